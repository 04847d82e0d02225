// Symmetric inter-level Newtonian pass (Eq. force-newton-inter, both lines at once): for two
// disjoint lists A and B, every pair (i in A, j in B) is evaluated once and gives both
//   a_i += G m_j x_ji / r^3      (A due to B)      and      a_j -= G m_i x_ji / r^3   (B due to A),
// the pairwise kicks of kick_sf in Algorithm hhs-fsi.  The two one-sided passes evaluate
// every pair twice; here the separation, r^2 and r^-3 are formed once and only the two
// weightings and sums differ.
//
// Work decomposition.  A 2-D grid: blockIdx.y over contiguous chunks of B (j-splits, as in
// the one-sided kernels), blockIdx.x over groups of A's i-blocks (a block takes the i-blocks
// g, g + ngroups, ... of the group g).  The i-side sums stay in registers and are written per
// (i-block, split) like the one-sided partials.  The j-side of a pair needs a reduction over
// the block's i-particles, done in a fixed order, so results are deterministic:
//   - each lane sums its own two i-particles' terms for 8 consecutive sources;
//   - a warp reduce-scatter (shuffles by 16, 8, 4, then 2 and 1) leaves the warp sum of
//     source s on the lanes 4s .. 4s + 3 (9 shuffles and 9 adds per component for 8 sources,
//     instead of 5 per source for a plain butterfly);
//   - the four warps' sums of a tile are added in order, and the block adds each tile's sums
//     in FP64 into its partials pj[group][c][j] (one group owns each (group, j) element).
// The finalisation sums the i-side partials over the splits and the j-side partials over the
// groups (launch_finalize_vec, the latter with the scale -G).
//
// Mixed precision: float-float separations and FP32 pair arithmetic as in the fast one-sided
// pass, packed f32x2 over the thread's two i-particles, compensated folds of the i-side sums
// every 64 sources, FP32 tree sums of 256 terms for the j-side of a tile.  FP64 mode: the same
// layout with one i-particle a thread and FP64 arithmetic.
#include "pair_bodies.cuh"

namespace frost {
namespace {

using namespace dev;

constexpr int SYM_BS = 128;
constexpr int SYM_TJ = 128;
constexpr int SYM_WARPS = SYM_BS / 32;
// a stand-in for the sources past the end of a tile: zero mass, far from every particle
// (its r^-3 flushes to zero, so it adds nothing to either side)
constexpr float SYM_FAR = 1.0e15f;

// warp reduce-scatter of v[8] (8 sources): returns on lane l the warp sum of source
// (l >> 2) & 7; the order of the additions is fixed
template <class T>
__device__ __forceinline__ T reduce_scatter8(const T (&v)[8], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    T c1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T send = b4 ? v[k] : v[4 + k];
        const T keep = b4 ? v[4 + k] : v[k];
        c1[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    T c2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const T send = b3 ? c1[k] : c1[2 + k];
        const T keep = b3 ? c1[2 + k] : c1[k];
        c2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const T send = b2 ? c2[0] : c2[1];
    const T keep = b2 ? c2[1] : c2[0];
    T c3 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    c3 = c3 + __shfl_xor_sync(0xffffffffu, c3, 2);
    c3 = c3 + __shfl_xor_sync(0xffffffffu, c3, 1);
    return c3;
}

// One source (staged duplicated as in acc_x2_j) against the thread's two particles: the
// i-side terms m_j x_ji / r^3 into (ax, ay, az) and the j-side sum over the two particles of
// m_i x_ji / r^3 into (cx, cy, cz).
__device__ __forceinline__ void sym_x2_j(const float4 A, const float4 B, const float4 C, const float2 M,
                                         const AccX2I &P, const float2 mi, float2 e2, float2 &ax, float2 &ay,
                                         float2 &az, float &cx, float &cy, float &cz)
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), P.nxh), __fadd2_rn(make_float2(B.z, B.w), P.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), P.nyh), __fadd2_rn(make_float2(C.x, C.y), P.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), P.nzh), __fadd2_rn(make_float2(C.z, C.w), P.nzl));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 u = __fmul2_rn(ri, __fmul2_rn(ri, ri));  // r^-3
    const float2 w = __fmul2_rn(M, u);                      // m_j r^-3
    ax = __ffma2_rn(w, dx, ax);
    ay = __ffma2_rn(w, dy, ay);
    az = __ffma2_rn(w, dz, az);
    const float2 wj = __fmul2_rn(mi, u);                    // m_i r^-3
    cx = fmaf(wj.y, dx.y, wj.x * dx.x);
    cy = fmaf(wj.y, dy.y, wj.x * dy.x);
    cz = fmaf(wj.y, dz.y, wj.x * dz.x);
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_acc_sym_mixed(const float4 *__restrict__ irec, const float4 *__restrict__ jrec,
                                                      int n_a, int n_s, int nblk_i, int j_per_split, float eps2,
                                                      double *__restrict__ part, double *__restrict__ pj)
{
    constexpr int ILP = 2, W = BS / 32;
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ];
    __shared__ float2 sM[TJ];
    __shared__ float sJ[W][3][TJ];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x, ng = gridDim.x;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    const float2 e2 = make_float2(eps2, eps2);
    for (int ib = g; ib < nblk_i; ib += ng) {
        const int ibase = ib * BS * ILP;
        // the thread's two particles; past the end: zero mass, far from every source
        float4 a0 = make_float4(SYM_FAR, SYM_FAR, SYM_FAR, 0.f), a1 = a0, b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
        const int i0 = ibase + tid, i1 = ibase + BS + tid;
        if (i0 < n_a) {
            a0 = irec[i0];
            b0 = irec[n_a + i0];
        }
        if (i1 < n_a) {
            a1 = irec[i1];
            b1 = irec[n_a + i1];
        }
        AccX2I P;
        P.nxh = make_float2(-a0.x, -a1.x);
        P.nyh = make_float2(-a0.y, -a1.y);
        P.nzh = make_float2(-a0.z, -a1.z);
        P.nxl = make_float2(-b0.x, -b1.x);
        P.nyl = make_float2(-b0.y, -b1.y);
        P.nzl = make_float2(-b0.z, -b1.z);
        const float2 mi = make_float2(a0.w, a1.w);
        float hx[ILP] = {0.f, 0.f}, hy[ILP] = {0.f, 0.f}, hz[ILP] = {0.f, 0.f};
        float lx[ILP] = {0.f, 0.f}, ly[ILP] = {0.f, 0.f}, lz[ILP] = {0.f, 0.f};
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            const int cnt8 = (cnt + 7) & ~7;
            __syncthreads();
            for (int t = tid; t < cnt8; t += BS) {
                float4 a = make_float4(-SYM_FAR, -SYM_FAR, -SYM_FAR, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t < cnt) {
                    a = jrec[j0 + t];
                    b = jrec[n_s + j0 + t];
                }
                sA[t] = make_float4(a.x, a.x, a.y, a.y);
                sB[t] = make_float4(a.z, a.z, b.x, b.x);
                sC[t] = make_float4(b.y, b.y, b.z, b.z);
                sM[t] = make_float2(a.w, a.w);
            }
            __syncthreads();
            for (int c0 = 0; c0 < cnt8; c0 += 64) {
                const int c1 = min(cnt8, c0 + 64);
                float2 ax2 = make_float2(0.f, 0.f), ay2 = ax2, az2 = ax2;
                for (int jj = c0; jj < c1; jj += 8) {
                    float cx[8], cy[8], cz[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        sym_x2_j(sA[jj + u], sB[jj + u], sC[jj + u], sM[jj + u], P, mi, e2, ax2, ay2, az2, cx[u], cy[u],
                                 cz[u]);
                    const float rx = reduce_scatter8(cx, lane);
                    const float ry = reduce_scatter8(cy, lane);
                    const float rz = reduce_scatter8(cz, lane);
                    if ((lane & 3) == 0) {
                        const int s = jj + (lane >> 2);
                        sJ[warp][0][s] = rx;
                        sJ[warp][1][s] = ry;
                        sJ[warp][2][s] = rz;
                    }
                }
                fold2(hx[0], lx[0], ax2.x);
                fold2(hy[0], ly[0], ay2.x);
                fold2(hz[0], lz[0], az2.x);
                fold2(hx[1], lx[1], ax2.y);
                fold2(hy[1], ly[1], ay2.y);
                fold2(hz[1], lz[1], az2.y);
            }
            __syncthreads();
            // the tile's j-side sums over the block's 256 particles, added to the group's partials
            for (int t = tid; t < cnt; t += BS) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v = sJ[0][c][t];
#pragma unroll
                    for (int q = 1; q < W; ++q) v += sJ[q][c][t];
                    double *dst = pj + ((size_t)g * 3 + c) * n_s + j0 + t;
                    *dst = (ib == g) ? (double)v : *dst + (double)v;
                }
            }
        }
        // the i-side partials of this i-block for this split
        double *p = part + (size_t)blockIdx.y * 3 * n_a;
        if (i0 < n_a) {
            p[i0] = (double)hx[0] + (double)lx[0];
            p[n_a + i0] = (double)hy[0] + (double)ly[0];
            p[2 * n_a + i0] = (double)hz[0] + (double)lz[0];
        }
        if (i1 < n_a) {
            p[i1] = (double)hx[1] + (double)lx[1];
            p[n_a + i1] = (double)hy[1] + (double)ly[1];
            p[2 * n_a + i1] = (double)hz[1] + (double)lz[1];
        }
    }
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_acc_sym_fp64(const double4_32a *__restrict__ irec,
                                                     const double4_32a *__restrict__ jrec, int n_a, int n_s,
                                                     int nblk_i, int j_per_split, double eps2,
                                                     double *__restrict__ part, double *__restrict__ pj)
{
    constexpr int W = BS / 32;
    __shared__ double4_32a sJr[TJ];
    __shared__ double sJ[W][3][TJ];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x, ng = gridDim.x;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    for (int ib = g; ib < nblk_i; ib += ng) {
        const int i = ib * BS + tid;
        double4_32a I = make_double4_32a((double)SYM_FAR, (double)SYM_FAR, (double)SYM_FAR, 0.0);
        if (i < n_a) I = irec[i];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            const int cnt8 = (cnt + 7) & ~7;
            __syncthreads();
            for (int t = tid; t < cnt8; t += BS)
                sJr[t] = (t < cnt) ? jrec[j0 + t]
                                   : make_double4_32a(-(double)SYM_FAR, -(double)SYM_FAR, -(double)SYM_FAR, 0.0);
            __syncthreads();
            for (int jj = 0; jj < cnt8; jj += 8) {
                double cx[8], cy[8], cz[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const double4_32a J = sJr[jj + u];
                    const double dx = J.x - I.x, dy = J.y - I.y, dz = J.z - I.z;
                    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
                    const double ri = rsqrt(r2);
                    const double uu = ri * ri * ri;
                    const double w = J.w * uu;
                    ax = fma(w, dx, ax);
                    ay = fma(w, dy, ay);
                    az = fma(w, dz, az);
                    const double wj = I.w * uu;
                    cx[u] = wj * dx;
                    cy[u] = wj * dy;
                    cz[u] = wj * dz;
                }
                const double rx = reduce_scatter8(cx, lane);
                const double ry = reduce_scatter8(cy, lane);
                const double rz = reduce_scatter8(cz, lane);
                if ((lane & 3) == 0) {
                    const int s = jj + (lane >> 2);
                    sJ[warp][0][s] = rx;
                    sJ[warp][1][s] = ry;
                    sJ[warp][2][s] = rz;
                }
            }
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double v = sJ[0][c][t];
#pragma unroll
                    for (int q = 1; q < W; ++q) v += sJ[q][c][t];
                    double *dst = pj + ((size_t)g * 3 + c) * n_s + j0 + t;
                    *dst = (ib == g) ? v : *dst + v;
                }
            }
        }
        if (i < n_a) {
            double *p = part + (size_t)blockIdx.y * 3 * n_a;
            p[i] = ax;
            p[n_a + i] = ay;
            p[2 * n_a + i] = az;
        }
    }
}

template <typename K>
int sym_occupancy(K kernel)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, SYM_BS, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

}  // namespace

SymShape sym_shape(bool mixed, int n_a, int n_s, int n_sm, size_t part_elems, size_t pj_elems)
{
    static int occ[2] = {0, 0};
    int &o = occ[mixed ? 1 : 0];
    if (!o) o = mixed ? sym_occupancy(k_acc_sym_mixed<SYM_BS, SYM_TJ>) : sym_occupancy(k_acc_sym_fp64<SYM_BS, SYM_TJ>);
    SymShape sh;
    const int ipb = mixed ? 2 * SYM_BS : SYM_BS;
    sh.nblk_i = std::max(1, (n_a + ipb - 1) / ipb);
    const long long max_groups = std::max<long long>(1, (long long)(pj_elems / (3 * (size_t)std::max(n_s, 1))));
    const int per = (int)((sh.nblk_i + std::min<long long>(max_groups, 64) - 1) / std::min<long long>(max_groups, 64));
    sh.ngroups = (sh.nblk_i + per - 1) / per;
    // about four waves of blocks; each split at least one tile, partials within their buffer
    const long long cap = (long long)o * n_sm;
    const int tiles = (n_s + SYM_TJ - 1) / SYM_TJ;
    long long ns = (4 * cap + sh.ngroups - 1) / sh.ngroups;
    ns = std::min<long long>(ns, tiles);
    ns = std::min<long long>(ns, (long long)(part_elems / (3 * (size_t)std::max(n_a, 1))));
    ns = std::max<long long>(ns, 1);
    const int tps = (tiles + (int)ns - 1) / (int)ns;
    sh.j_per_split = tps * SYM_TJ;
    sh.nsplit = (n_s + sh.j_per_split - 1) / sh.j_per_split;
    sh.blocks_per_wave = (int)cap;
    return sh;
}

void launch_acc_sym(cudaStream_t s, bool mixed, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                    double *part, double *pj, const SymShape &sh)
{
    const dim3 grid(sh.ngroups, sh.nsplit);
    if (mixed)
        k_acc_sym_mixed<SYM_BS, SYM_TJ><<<grid, SYM_BS, 0, s>>>((const float4 *)irec, (const float4 *)jrec, n_a, n_s,
                                                                sh.nblk_i, sh.j_per_split, (float)eps2, part, pj);
    else
        k_acc_sym_fp64<SYM_BS, SYM_TJ><<<grid, SYM_BS, 0, s>>>((const double4_32a *)irec, (const double4_32a *)jrec,
                                                               n_a, n_s, sh.nblk_i, sh.j_per_split, eps2, part, pj);
}

}  // namespace frost
