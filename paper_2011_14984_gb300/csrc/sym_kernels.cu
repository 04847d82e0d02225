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
// double-float slots of the reduced (B) side of the symmetric gradient kick_sf passes, per
// (source, group of i-blocks, warp): 8 per source and group, as the 8 slots per particle and
// split of the one-sided passes
constexpr int SYM_BSLOTS = 2;
static_assert(SYM_WARPS == SYM_PCNT_WARPS, "pcnt is sized for SYM_PCNT_WARPS warps a block");

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

// the same for v[4] (4 sources): returns on lane l the warp sum of source (l >> 3) & 3
template <class T>
__device__ __forceinline__ T reduce_scatter4(const T (&v)[4], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8;
    T c1[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const T send = b4 ? v[k] : v[2 + k];
        const T keep = b4 ? v[2 + k] : v[k];
        c1[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    const T send = b3 ? c1[0] : c1[1];
    const T keep = b3 ? c1[1] : c1[0];
    T c2 = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    c2 = c2 + __shfl_xor_sync(0xffffffffu, c2, 4);
    c2 = c2 + __shfl_xor_sync(0xffffffffu, c2, 2);
    return c2 + __shfl_xor_sync(0xffffffffu, c2, 1);
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

template <int BS, int TJ>
__global__ void k_acc_sym_defer_mixed(const float4 *__restrict__ irec, const float4 *__restrict__ jrec, int n_a,
                                      int n_s, int nblk_i, int j_per_split, float eps2, double eps2d,
                                      const float *__restrict__ wA, const float *__restrict__ wB,
                                      const int32_t *__restrict__ ilist, const int32_t *__restrict__ jlist,
                                      const double *__restrict__ mstore, double *__restrict__ part,
                                      double *__restrict__ pj, uint8_t *__restrict__ pcnt);
template <int BS, int TJ>
__global__ void k_grad_sym_mixed(const float4 *__restrict__ irec, const float4 *__restrict__ jrec, int n_a, int n_s,
                                 int nblk_i, int j_per_split, double eps2d, const float *__restrict__ wA,
                                 const float *__restrict__ wB, double *__restrict__ part, double *__restrict__ pj,
                                 uint8_t *__restrict__ pcnt);

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

SymShape sym_shape(int kind, int n_a, int n_s, int n_sm, size_t part_elems, size_t pj_elems)
{
    static int occ[SYM_KINDS] = {0, 0, 0, 0};
    int &o = occ[kind];
    if (!o) {
        switch (kind) {
        case SYM_ACC_FP64: o = sym_occupancy(k_acc_sym_fp64<SYM_BS, SYM_TJ>); break;
        case SYM_ACC_DEFER: o = sym_occupancy(k_acc_sym_defer_mixed<SYM_BS, SYM_TJ>); break;
        case SYM_GRAD: o = sym_occupancy(k_grad_sym_mixed<SYM_BS, SYM_TJ>); break;
        default: o = sym_occupancy(k_acc_sym_mixed<SYM_BS, SYM_TJ>); break;
        }
    }
    SymShape sh;
    const int ipb = (kind == SYM_ACC_FP64) ? SYM_BS : 2 * SYM_BS;
    sh.nblk_i = std::max(1, (n_a + ipb - 1) / ipb);
    const long long max_groups = std::max<long long>(1, (long long)(pj_elems / (3 * (size_t)std::max(n_s, 1))));
    const int per = (int)((sh.nblk_i + std::min<long long>(max_groups, 64) - 1) / std::min<long long>(max_groups, 64));
    sh.ngroups = (sh.nblk_i + per - 1) / per;
    // The split count.  Every block takes the same number of i-blocks, so its work is about
    // its tiles per split (plus a quarter tile of fixed work); an SM runs up to o blocks at a
    // time and its share of the grid, ceil(blocks / n_sm) blocks, sets the kernel's time:
    // cost = share x (tiles + 1/4) / min(share, o).  The count minimises it, with the partials
    // within their buffer; among equal costs the fewest splits.
    const long long cap = (long long)o * n_sm;
    const int tiles = (n_s + SYM_TJ - 1) / SYM_TJ;
    long long ns_max = std::min<long long>(tiles, (long long)(part_elems / (3 * (size_t)std::max(n_a, 1))));
    ns_max = std::max<long long>(ns_max, 1);
    double best = -1.0;
    int best_tps = tiles;
    for (long long ns = 1; ns <= ns_max; ++ns) {
        const int tps = (int)((tiles + ns - 1) / ns);
        const long long nsplit = (tiles + tps - 1) / tps;
        const long long share = (sh.ngroups * nsplit + n_sm - 1) / n_sm;
        const double cost = (double)share * (tps + 0.25) / (double)std::min<long long>(share, o);
        if (best < 0.0 || cost < best - 1e-9) {
            best = cost;
            best_tps = tps;
        }
    }
    sh.j_per_split = best_tps * SYM_TJ;
    sh.nsplit = (n_s + sh.j_per_split - 1) / sh.j_per_split;
    sh.blocks_per_wave = (int)cap;
    sh.max_blocks = (long long)sh.ngroups * ns_max;
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

// ======================================================================================
// Symmetric time-step pass over one set (Sec. 4.3, tau_i = min_j of the symmetrised pair
// time-steps).  The pair criteria are symmetric bit for bit: x_ij = -x_ji and v_ij = -v_ji
// exactly in IEEE arithmetic, r^2, v^2, r.v are the same sums of the same products, and
// G (m_i + m_j) is a commutative sum.  So every pair can be evaluated once for both particles.
// A minimum is exact and independent of the order, so the j side needs no fixed-order sum:
// a warp reduce-scatter of the minima of 8 sources, a shared-memory atomicMin per warp and a
// global atomicMin per source and block (non-negative floats order as their bit patterns).
//
// Tiles: row ib (the i-block of 256 particles) takes the tiles from its own range onwards;
// the two tiles that overlap its own particles run the one-sided masked loop (i side only:
// their particles are also this block's i-particles), the later ones the symmetric loop.
// A criterion is skipped only when it can lower neither particle's minimum: the bound is the
// larger of the i-particle's running bound and the source's bound read from the global minima
// when the tile is staged (stale values are larger, so the test stays conservative).  The
// result is the exact minimum over all pairs, the same bits as the one-sided pass.
// ======================================================================================
namespace frost {
namespace {

using namespace dev;

// One source against the thread's two particles (as tstep_x2_j), with the skip bound
// max(bnd_i, bnd_j); tj[k]: the pair's time-step if evaluated for lane k, else +inf.
// valid = false: a stand-in past the end of the list (no update, +inf).
template <int SYM>
__device__ __forceinline__ void tstep_sym_x2_j(const float4 A, const float4 B, const float4 C, const float4 V0,
                                               const float4 V1, const float4 W0, const float4 W1, const TstepX2I &P,
                                               float eta, float eta15, float bndj, bool valid, float (&best)[2],
                                               float (&minr2)[2], float (&bnd)[2], float (&tj)[2])
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), P.nxh), __fadd2_rn(make_float2(B.z, B.w), P.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), P.nyh), __fadd2_rn(make_float2(C.x, C.y), P.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), P.nzh), __fadd2_rn(make_float2(C.z, C.w), P.nzl));
    const float2 ux = __fadd2_rn(make_float2(V0.x, V0.y), P.nvx);
    const float2 uy = __fadd2_rn(make_float2(V0.z, V0.w), P.nvy);
    const float2 uz = __fadd2_rn(make_float2(V1.x, V1.y), P.nvz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float2 v2 = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __fmul2_rn(uz, uz)));
    const float2 rv = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
    const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 gm = __fadd2_rn(P.gm, make_float2(V1.z, V1.w));
    const float2 q = __fmul2_rn(__fmul2_rn(gm, ri2), ri);
    const float2 tff = make_float2(rsqrtf(q.x), rsqrtf(q.y));
    const float2 rvr2 = __fmul2_rn(rv, ri2);
    const float2 iv = make_float2(rsqrtf(v2.x), rsqrtf(v2.y));
    const float2 tfb = __fmul2_rn(__fmul2_rn(r2, ri), iv);
    const float Bb[2] = {fmaxf(bnd[0], bndj), fmaxf(bnd[1], bndj)};
    const float2 ce = make_float2(Bb[0] * eta, Bb[1] * eta);
    const float2 z = __fmul2_rn(ce, rvr2);
    float2 hfb, mfb;
    if (SYM & 4) {
        const float2 wx = __fadd2_rn(make_float2(W0.x, W0.y), P.nax);
        const float2 wy = __fadd2_rn(make_float2(W0.z, W0.w), P.nay);
        const float2 wz = __fadd2_rn(make_float2(W1.x, W1.y), P.naz);
        const float2 va = __ffma2_rn(ux, wx, __ffma2_rn(uy, wy, __fmul2_rn(uz, wz)));
        const float2 niv2 = __fmul2_rn(__fmul2_rn(make_float2(-1.f, -1.f), iv), iv);
        hfb = __ffma2_rn(va, niv2, rvr2);
        const float2 zb = __fmul2_rn(ce, hfb);
        mfb = make_float2(-fabsf(zb.x), -fabsf(zb.y));
    } else {
        hfb = __ffma2_rn(__fmul2_rn(gm, ri), __fmul2_rn(iv, iv), make_float2(1.f, 1.f));
        mfb = make_float2(-fabsf(z.x) * hfb.x, -fabsf(z.y) * hfb.y);
    }
    const float2 mff = make_float2(-1.5f * fabsf(z.x), -1.5f * fabsf(z.y));
    const float2 lff = __ffma2_rn(mff, tff, tff);
    const float2 lfb = __ffma2_rn(mfb, tfb, tfb);
    const float tf[2] = {tff.x, tff.y}, tb[2] = {tfb.x, tfb.y}, rq[2] = {rvr2.x, rvr2.y}, hq[2] = {hfb.x, hfb.y};
    const float rr[2] = {r2.x, r2.y}, vv[2] = {v2.x, v2.y}, lf[2] = {lff.x, lff.y}, lb[2] = {lfb.x, lfb.y};
    bool nff[2], nfb[2];
    bool any = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (valid) minr2[k] = fminf(minr2[k], rr[k]);
        nff[k] = valid && !(lf[k] >= Bb[k]);
        nfb[k] = valid && (vv[k] > 0.f) && !(lb[k] >= Bb[k]);
        any = any || nff[k] || nfb[k];
        tj[k] = INFINITY;
    }
    if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float t = INFINITY;
            if (nff[k]) t = tf[k] * symf<(SYM & 3)>(eta15 * rq[k] * tf[k]);
            if (nfb[k]) {
                const float dfb = (SYM & 4) ? eta * hq[k] * tb[k] : eta * rq[k] * hq[k] * tb[k];
                t = fminf(t, tb[k] * symf<(SYM & 3)>(dfb));
            }
            tj[k] = t;
            best[k] = fminf(best[k], t);
            bnd[k] = 1.001f * best[k];
        }
    }
}

__device__ __forceinline__ float reduce_scatter8_min(const float (&v)[8], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float c1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? v[k] : v[4 + k];
        const float keep = b4 ? v[4 + k] : v[k];
        c1[k] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
    float c2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? c1[k] : c1[2 + k];
        const float keep = b3 ? c1[2 + k] : c1[k];
        c2[k] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 8));
    }
    const float send = b2 ? c2[0] : c2[1];
    const float keep = b2 ? c2[1] : c2[0];
    float c3 = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 4));
    c3 = fminf(c3, __shfl_xor_sync(0xffffffffu, c3, 2));
    return fminf(c3, __shfl_xor_sync(0xffffffffu, c3, 1));
}

constexpr unsigned kInfBits = 0x7f800000u;

__global__ void k_fill_inf(unsigned *__restrict__ p, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = kInfBits;
}

template <int BS, int TJ, int SYM>
__global__ void __launch_bounds__(BS) k_tstep_sym_mixed(const float4 *__restrict__ rec, int n, int ntiles, int tps,
                                                        float eta, double *__restrict__ part,
                                                        unsigned *__restrict__ jbest, int *__restrict__ err)
{
    constexpr int ILP = 2;
    constexpr int TA = (SYM & 4) ? TJ : 1;
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ], sV0[TJ], sV1[TJ];
    __shared__ float4 sW0[TA], sW1[TA];
    __shared__ float sBj[TJ];
    __shared__ unsigned sJ[TJ];
    const int tid = threadIdx.x, lane = tid & 31;
    // block -> (row, split) of the upper triangle of tiles
    const int nblk = (n + BS * ILP - 1) / (BS * ILP);
    int b = blockIdx.x, ib = 0;
    for (; ib < nblk; ++ib) {
        const int S = max(0, (ntiles - 2 * ib + tps - 1) / tps);
        if (b < S) break;
        b -= S;
    }
    if (ib >= nblk) return;
    const int ibase = ib * BS * ILP;
    const int tile0 = 2 * ib + b * tps, tile1 = min(ntiles, tile0 + tps);
    TstepMixedI<ILP> I;
    int ipos[ILP];
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + tid;
        ipos[k] = i;
        float4 a = make_float4(0.f, 0.f, 0.f, 1.f), bb = zero4, c = a, d = zero4;
        if (i < n) {
            a = rec[i];
            bb = rec[n + i];
            c = rec[2 * n + i];
            if (SYM & 4) d = rec[3 * n + i];
        }
        I.xh[k] = a.x; I.yh[k] = a.y; I.zh[k] = a.z;
        I.xl[k] = bb.x; I.yl[k] = bb.y; I.zl[k] = bb.z;
        I.vx[k] = c.x; I.vy[k] = c.y; I.vz[k] = c.z; I.gm[k] = c.w;
        I.ax[k] = d.x; I.ay[k] = d.y; I.az[k] = d.z;
    }
    // particles past the end take part in nothing (the bounds below keep them at +inf)
    const bool live[2] = {ipos[0] < n, ipos[1] < n};
    TstepX2I P;
    P.nxh = make_float2(-I.xh[0], -I.xh[1]);
    P.nyh = make_float2(-I.yh[0], -I.yh[1]);
    P.nzh = make_float2(-I.zh[0], -I.zh[1]);
    P.nxl = make_float2(-I.xl[0], -I.xl[1]);
    P.nyl = make_float2(-I.yl[0], -I.yl[1]);
    P.nzl = make_float2(-I.zl[0], -I.zl[1]);
    P.nvx = make_float2(-I.vx[0], -I.vx[1]);
    P.nvy = make_float2(-I.vy[0], -I.vy[1]);
    P.nvz = make_float2(-I.vz[0], -I.vz[1]);
    P.gm = make_float2(I.gm[0], I.gm[1]);
    P.nax = make_float2(-I.ax[0], -I.ax[1]);
    P.nay = make_float2(-I.ay[0], -I.ay[1]);
    P.naz = make_float2(-I.az[0], -I.az[1]);
    float best[2] = {INFINITY, INFINITY}, minr2[2] = {INFINITY, INFINITY}, bnd[2] = {INFINITY, INFINITY};
    const float eta15 = 1.5f * eta;
    for (int tile = tile0; tile < tile1; ++tile) {
        const int j0 = tile * TJ;
        const int cnt = min(TJ, n - j0);
        const int cnt8 = (cnt + 7) & ~7;
        const bool diag = tile < 2 * ib + 2;
        __syncthreads();
        for (int t = tid; t < cnt8; t += BS) {
            float4 a = zero4, bb = zero4, v = zero4;
            if (t < cnt) {
                a = rec[j0 + t];
                bb = rec[n + j0 + t];
                v = rec[2 * n + j0 + t];
            }
            sA[t] = make_float4(a.x, a.x, a.y, a.y);
            sB[t] = make_float4(a.z, a.z, bb.x, bb.x);
            sC[t] = make_float4(bb.y, bb.y, bb.z, bb.z);
            sV0[t] = make_float4(v.x, v.x, v.y, v.y);
            sV1[t] = make_float4(v.z, v.z, v.w, v.w);
            if (SYM & 4) {
                const float4 w = (t < cnt) ? rec[3 * n + j0 + t] : zero4;
                sW0[t] = make_float4(w.x, w.x, w.y, w.y);
                sW1[t] = make_float4(w.z, w.z, 0.f, 0.f);
            }
            sBj[t] = (t < cnt && !diag) ? 1.001f * __uint_as_float(jbest[j0 + t]) : INFINITY;
            sJ[t] = kInfBits;
        }
        __syncthreads();
        if (diag) {
            // the tiles of the block's own particles: every pair from the i side, masked i = j
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 a = sA[jj], bq = sB[jj], c = sC[jj], v0 = sV0[jj], v1 = sV1[jj];
                const float4 J0 = make_float4(a.x, a.z, bq.x, 0.f);
                const float4 J1 = make_float4(bq.z, c.x, c.z, 0.f);
                const float4 JV = make_float4(v0.x, v0.z, v1.x, v1.z);
                float4 JA = zero4;
                if (SYM & 4) JA = make_float4(sW0[jj].x, sW0[jj].z, sW1[jj].x, 0.f);
                tstep_mixed_j<ILP, SYM, true>(J0, J1, JV, JA, I, eta, eta15, j0 + jj, ipos, best, minr2);
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) bnd[k] = 1.001f * best[k];
            continue;
        }
        for (int jj = 0; jj < cnt8; jj += 8) {
            float tmin[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float tj[2];
                tstep_sym_x2_j<SYM>(sA[jj + u], sB[jj + u], sC[jj + u], sV0[jj + u], sV1[jj + u],
                                    (SYM & 4) ? sW0[jj + u] : zero4, (SYM & 4) ? sW1[jj + u] : zero4, P, eta, eta15,
                                    sBj[jj + u], jj + u < cnt, best, minr2, bnd, tj);
                tmin[u] = fminf(live[0] ? tj[0] : INFINITY, live[1] ? tj[1] : INFINITY);
            }
            const float m = reduce_scatter8_min(tmin, lane);
            if ((lane & 3) == 0 && m < INFINITY) atomicMin(&sJ[jj + (lane >> 2)], __float_as_uint(m));
        }
        __syncthreads();
        for (int t = tid; t < cnt; t += BS)
            if (sJ[t] < kInfBits) atomicMin(&jbest[j0 + t], sJ[t]);
    }
    // the i side of this row and split
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        if (!live[k]) continue;
        part[(size_t)b * n + ipos[k]] = (double)best[k];
        if (minr2[k] == 0.f) atomicOr(err, ERR_COINCIDENT);
    }
}

__global__ void k_finalize_tau_sym(const double *__restrict__ part, const unsigned *__restrict__ jbest, int n,
                                   int ntiles, int tps, int ipb, double eta, double *__restrict__ tau,
                                   int *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ib = i / ipb;
    const int S = max(0, (ntiles - 2 * ib + tps - 1) / tps);
    double b = (double)__uint_as_float(jbest[i]);
    for (int s = 0; s < S; ++s) b = fmin(b, part[(size_t)s * n + i]);
    const double t = eta * b;
    if (!(t > 0.0)) atomicOr(err, ERR_NONFINITE);
    tau[i] = t;
}

}  // namespace

TstepSymShape tstep_sym_shape(int n, int n_sm, size_t part_elems)
{
    TstepSymShape sh;
    constexpr int BS = SYM_BS, ILP = 2, TJ = SYM_TJ;
    const int nblk = (n + BS * ILP - 1) / (BS * ILP);
    sh.ntiles = (n + TJ - 1) / TJ;
    // about 8 waves of blocks (6 per SM), each at least one tile, the row-0 partials in part
    const long long tiles_total = (long long)nblk * sh.ntiles - (long long)nblk * (nblk - 1);  // upper triangle
    const long long target = 8LL * 6 * n_sm;
    int tps = (int)std::max<long long>(1, (tiles_total + target - 1) / target);
    while ((long long)((sh.ntiles + tps - 1) / tps) * n > (long long)part_elems) ++tps;
    sh.tps = tps;
    long long blocks = 0;
    for (int ib = 0; ib < nblk; ++ib) blocks += std::max(0, (sh.ntiles - 2 * ib + tps - 1) / tps);
    sh.blocks = (int)blocks;
    return sh;
}

void launch_tstep_sym(cudaStream_t s, const void *rec, int n, double eta, int sym, const TstepSymShape &sh,
                      double *part, unsigned *jbest, double *tau, int *err)
{
    k_fill_inf<<<(n + 255) / 256, 256, 0, s>>>(jbest, n);
#define FROST_TSTEP_SYM_CASE(SYMV)                                                                       \
    k_tstep_sym_mixed<SYM_BS, SYM_TJ, SYMV><<<sh.blocks, SYM_BS, 0, s>>>((const float4 *)rec, n, sh.ntiles, sh.tps, \
                                                                         (float)eta, part, jbest, err);
    switch (sym) {
    case 0: FROST_TSTEP_SYM_CASE(0) break;
    case 1: FROST_TSTEP_SYM_CASE(1) break;
    case 4: FROST_TSTEP_SYM_CASE(4) break;
    case 5: FROST_TSTEP_SYM_CASE(5) break;
    case 6: FROST_TSTEP_SYM_CASE(6) break;
    default: FROST_TSTEP_SYM_CASE(2) break;
    }
#undef FROST_TSTEP_SYM_CASE
    k_finalize_tau_sym<<<(n + 255) / 256, 256, 0, s>>>(part, jbest, n, sh.ntiles, sh.tps, 2 * SYM_BS, eta, tau, err);
}

}  // namespace frost

// ======================================================================================
// Symmetric prepass of the Newtonian pass that feeds a gradient: wmax_i = max_j m_j / r^3 =
// (min_j r^2 m_j^(-2/3))^(-3/2).  r^2 is symmetric bit for bit and m^(-2/3) is a function of
// the particle's own record, so each pair gives both particles' values; the minimum (and the
// monotone map to wmax, then integer atomicMax on the float bits) is exact and independent
// of the order, so the result is the one-sided prepass's, bit for bit.
// ======================================================================================
namespace frost {
namespace {

using namespace dev;

__device__ __forceinline__ float mq_of(float m) { return (m > 0.f) ? exp2f(-0.6666667f * log2f(m)) : INFINITY; }
__device__ __forceinline__ float wmax_of(float q)
{
    const float y = rsqrtf(q);
    return y * y * y;
}

// stage a tile of source records (duplicated for the packed loop) with m^(-2/3); past cnt:
// far, massless stand-ins
__device__ __forceinline__ void wsym_stage(const float4 *__restrict__ jrec, int n_s, int j0, int cnt, int cnt8,
                                           float4 *sA, float4 *sB, float4 *sC, float2 *sM, unsigned *sQ)
{
    for (int t = threadIdx.x; t < cnt8; t += blockDim.x) {
        float4 a = make_float4(-SYM_FAR, -SYM_FAR, -SYM_FAR, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < cnt) {
            a = jrec[j0 + t];
            b = jrec[n_s + j0 + t];
        }
        const float mq = (t < cnt) ? mq_of(a.w) : INFINITY;
        sA[t] = make_float4(a.x, a.x, a.y, a.y);
        sB[t] = make_float4(a.z, a.z, b.x, b.x);
        sC[t] = make_float4(b.y, b.y, b.z, b.z);
        sM[t] = make_float2(mq, mq);
        sQ[t] = kInfBits;
    }
}

// the off-diagonal loop over a staged tile: i side into qm, j side into sQ (minima of q)
__device__ __forceinline__ void wsym_tile(const float4 *sA, const float4 *sB, const float4 *sC, const float2 *sM,
                                          unsigned *sQ, int cnt8, const AccX2I &P, float2 mqi, float2 e2, float2 &qm,
                                          int lane)
{
    for (int jj = 0; jj < cnt8; jj += 8) {
        float qj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 A = sA[jj + u], B = sB[jj + u], C = sC[jj + u];
            const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), P.nxh), __fadd2_rn(make_float2(B.z, B.w), P.nxl));
            const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), P.nyh), __fadd2_rn(make_float2(C.x, C.y), P.nyl));
            const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), P.nzh), __fadd2_rn(make_float2(C.z, C.w), P.nzl));
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
            const float2 q = __fmul2_rn(r2, sM[jj + u]);
            qm.x = fminf(qm.x, q.x);
            qm.y = fminf(qm.y, q.y);
            const float2 qs = __fmul2_rn(r2, mqi);
            qj[u] = fminf(qs.x, qs.y);
        }
        const float m = reduce_scatter8_min(qj, lane);
        if ((lane & 3) == 0 && m < INFINITY) atomicMin(&sQ[jj + (lane >> 2)], __float_as_uint(m));
    }
}

__device__ __forceinline__ void wsym_load_i(const float4 *__restrict__ irec, int n_a, int ibase, int bs, AccX2I &P,
                                            float2 &mqi, bool (&live)[2], AccMixedI<2> &I)
{
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = ibase + k * bs + threadIdx.x;
        live[k] = i < n_a;
        float4 a = make_float4(SYM_FAR, SYM_FAR, SYM_FAR, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live[k]) {
            a = irec[i];
            b = irec[n_a + i];
        }
        I.xh[k] = a.x; I.yh[k] = a.y; I.zh[k] = a.z;
        I.xl[k] = b.x; I.yl[k] = b.y; I.zl[k] = b.z;
        (k == 0 ? mqi.x : mqi.y) = live[k] ? mq_of(a.w) : INFINITY;
    }
    P.nxh = make_float2(-I.xh[0], -I.xh[1]);
    P.nyh = make_float2(-I.yh[0], -I.yh[1]);
    P.nzh = make_float2(-I.zh[0], -I.zh[1]);
    P.nxl = make_float2(-I.xl[0], -I.xl[1]);
    P.nyl = make_float2(-I.yl[0], -I.yl[1]);
    P.nzl = make_float2(-I.zl[0], -I.zl[1]);
}

// one set, upper triangle of tiles (rows and parts as in k_tstep_sym_mixed)
template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_wmax_sym_self(const float4 *__restrict__ rec, int n, int ntiles, int tps,
                                                      float eps2, float *__restrict__ wmax)
{
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ];
    __shared__ float2 sM[TJ];
    __shared__ unsigned sQ[TJ];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nblk = (n + 2 * BS - 1) / (2 * BS);
    int b = blockIdx.x, ib = 0;
    for (; ib < nblk; ++ib) {
        const int S = max(0, (ntiles - 2 * ib + tps - 1) / tps);
        if (b < S) break;
        b -= S;
    }
    if (ib >= nblk) return;
    const int ibase = ib * 2 * BS;
    const int tile0 = 2 * ib + b * tps, tile1 = min(ntiles, tile0 + tps);
    AccX2I P;
    AccMixedI<2> I;
    float2 mqi;
    bool live[2];
    wsym_load_i(rec, n, ibase, BS, P, mqi, live, I);
    const int ipos[2] = {ibase + tid, ibase + BS + tid};
    const float2 e2 = make_float2(eps2, eps2);
    float2 qm = make_float2(INFINITY, INFINITY);
    for (int tile = tile0; tile < tile1; ++tile) {
        const int j0 = tile * TJ, cnt = min(TJ, n - j0), cnt8 = (cnt + 7) & ~7;
        const bool diag = tile < 2 * ib + 2;
        __syncthreads();
        wsym_stage(rec, n, j0, cnt, cnt8, sA, sB, sC, sM, sQ);
        __syncthreads();
        if (diag) {
            // the block's own particles: the one-sided masked loop (the i side only)
            float w[2] = {qm.x, qm.y};
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 A = sA[jj], Bq = sB[jj], C = sC[jj];
                const float4 J0 = make_float4(A.x, A.z, Bq.x, 0.f);
                const float4 J1 = make_float4(Bq.z, C.x, C.z, sM[jj].x);
                wmax_mixed_j<2, true>(J0, J1, I, eps2, j0 + jj, ipos, w);
            }
            qm = make_float2(w[0], w[1]);
            continue;
        }
        wsym_tile(sA, sB, sC, sM, sQ, cnt8, P, mqi, e2, qm, lane);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS)
            if (sQ[t] < kInfBits) atomicMax((int *)&wmax[j0 + t], __float_as_int(wmax_of(__uint_as_float(sQ[t]))));
    }
    if (live[0]) atomicMax((int *)&wmax[ipos[0]], __float_as_int(wmax_of(qm.x)));
    if (live[1]) atomicMax((int *)&wmax[ipos[1]], __float_as_int(wmax_of(qm.y)));
}

// two disjoint lists: A on the register side (blocks of 256 along blockIdx.x), B reduced
// (chunks of j_per_split along blockIdx.y); wA, wB: the two lists' maxima (zeroed before)
template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_wmax_sym_cross(const float4 *__restrict__ irec, const float4 *__restrict__ jrec,
                                                       int n_a, int n_s, int j_per_split, float eps2,
                                                       float *__restrict__ wA, float *__restrict__ wB)
{
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ];
    __shared__ float2 sM[TJ];
    __shared__ unsigned sQ[TJ];
    const int tid = threadIdx.x, lane = tid & 31;
    const int ibase = blockIdx.x * 2 * BS;
    const int jb = blockIdx.y * j_per_split, je = min(n_s, jb + j_per_split);
    AccX2I P;
    AccMixedI<2> I;
    float2 mqi;
    bool live[2];
    wsym_load_i(irec, n_a, ibase, BS, P, mqi, live, I);
    const float2 e2 = make_float2(eps2, eps2);
    float2 qm = make_float2(INFINITY, INFINITY);
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0), cnt8 = (cnt + 7) & ~7;
        __syncthreads();
        wsym_stage(jrec, n_s, j0, cnt, cnt8, sA, sB, sC, sM, sQ);
        __syncthreads();
        wsym_tile(sA, sB, sC, sM, sQ, cnt8, P, mqi, e2, qm, lane);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS)
            if (sQ[t] < kInfBits) atomicMax((int *)&wB[j0 + t], __float_as_int(wmax_of(__uint_as_float(sQ[t]))));
    }
    if (live[0]) atomicMax((int *)&wA[ibase + tid], __float_as_int(wmax_of(qm.x)));
    if (live[1]) atomicMax((int *)&wA[ibase + BS + tid], __float_as_int(wmax_of(qm.y)));
}

}  // namespace

void launch_wmax_sym_self(cudaStream_t s, const void *rec, int n, double eps2, int n_sm, size_t part_elems,
                          float *wmax)
{
    cudaMemsetAsync(wmax, 0, sizeof(float) * n, s);
    const TstepSymShape sh = tstep_sym_shape(n, n_sm, part_elems);
    k_wmax_sym_self<SYM_BS, SYM_TJ><<<sh.blocks, SYM_BS, 0, s>>>((const float4 *)rec, n, sh.ntiles, sh.tps,
                                                                  (float)eps2, wmax);
}

void launch_wmax_sym_cross(cudaStream_t s, const void *recA, int nA, const void *recB, int nB, double eps2, int n_sm,
                           float *wA, float *wB)
{
    cudaMemsetAsync(wA, 0, sizeof(float) * nA, s);
    cudaMemsetAsync(wB, 0, sizeof(float) * nB, s);
    // the longer list on the register side; about 8 waves of 128-thread blocks (6 per SM)
    const bool swap = nB > nA;
    const int ni = swap ? nB : nA, nj = swap ? nA : nB;
    const int nblk = (ni + 2 * SYM_BS - 1) / (2 * SYM_BS);
    const int tiles = (nj + SYM_TJ - 1) / SYM_TJ;
    const long long target = 8LL * 6 * n_sm;
    const int ns = (int)std::max<long long>(1, std::min<long long>(tiles, (target + nblk - 1) / nblk));
    const int jps = ((tiles + ns - 1) / ns) * SYM_TJ;
    const dim3 grid(nblk, (nj + jps - 1) / jps);
    k_wmax_sym_cross<SYM_BS, SYM_TJ><<<grid, SYM_BS, 0, s>>>((const float4 *)(swap ? recB : recA),
                                                             (const float4 *)(swap ? recA : recB), ni, nj, jps,
                                                             (float)eps2, swap ? wB : wA, swap ? wA : wB);
}

}  // namespace frost

// ======================================================================================
// Symmetric passes of the gradient kick_sf (mixed precision): the Newtonian pass that feeds
// the gradient and the gradient itself, for two disjoint lists A (the register side) and B
// (the reduced side), each pair once for both lists (Eq. force-newton-inter and Eqs.
// force-gradient-inter-1/2, both lines).  The B-side term of a pair is the A-side term with
// the other mass and the opposite sign: x_ij = -x_ji, a_ij = -a_ji, and the gradient pair
// term r^-3 (a - 3 (x.a) x / r^2) is odd in (x, a).  The work decomposition and the fixed-order
// reduction of the B side are those of k_acc_sym_mixed; the B-side partials carry the
// receiver's sign (pj = sum over i of the terms of j due to i), so both sides finalise alike.
//
// Dominant terms, per side as in the one-sided passes.  A pair whose weight m_j r^-3 exceeds
// SLOT_FRACTION x wmax_i goes to one of i's deferred slots (up to GRAD_SLOTS a split); one
// whose m_i r^-3 exceeds SLOT_FRACTION x wmax_j is deferred for j, up to SYM_BSLOTS per
// (source, group, warp) in the order of the warp's ballots (their counts persist across the
// group's i-blocks in pcnt).  A deferred side adds nothing to the FP32 sums and takes its term
// in double-float: the A side after its split, per thread from the slots; the B side after
// each tile, from the ballots of the deferred pairs, read in a fixed order (warp, particle
// slot, lane) by the thread that owns the source.  So the B side is deterministic too.
// ======================================================================================
namespace frost {
namespace {

using namespace dev;

// Staging of the B-side state of tile entry t (cnt live sources from j0) for every warp: the
// warp's slots used so far for the source in this group (pcnt, zero on the group's first
// i-block), its threshold (SLOT_FRACTION wmax_j while slots are left, else +inf, as for the
// stand-ins past the end of the tile) and cleared ballot rows.
__device__ __forceinline__ void stage_bside(float (*sT)[SYM_TJ], int (*sCnt)[SYM_TJ], unsigned (*sQ)[2][SYM_TJ],
                                            const uint8_t *__restrict__ pcnt, int t, int cnt, int j0, int n_s, int g,
                                            bool first, float tj)
{
#pragma unroll
    for (int w = 0; w < SYM_WARPS; ++w) {
        int used = SYM_BSLOTS;
        if (t < cnt) used = first ? 0 : (int)pcnt[((size_t)g * SYM_WARPS + w) * n_s + j0 + t];
        sCnt[w][t] = used;
        sT[w][t] = (used < SYM_BSLOTS) ? tj : INFINITY;
        sQ[w][0][t] = sQ[w][1][t] = 0u;
    }
}

// The B side's dominant terms, per warp: at most SYM_BSLOTS of them for each (source, group
// of the block, warp), the first candidates in the order (particle slot k, lane); the others
// stay in the FP32 sums, as the candidates beyond a one-sided pass's slots do.  d0, d1: the
// lane's candidates on entry, the deferred ones on return; cnt: the slots the warp has used
// for this source (shared memory); q0, q1: the ballots of the deferred pairs.
__device__ __forceinline__ void bside_defer(bool &d0, bool &d1, int *cnt, unsigned *q0, unsigned *q1, int lane)
{
    if (!__any_sync(0xffffffffu, d0 || d1)) return;
    const unsigned m0 = __ballot_sync(0xffffffffu, d0), m1 = __ballot_sync(0xffffffffu, d1);
    const int avail = SYM_BSLOTS - *cnt;
    const unsigned lt = (1u << lane) - 1u;
    d0 = d0 && (__popc(m0 & lt) < avail);
    d1 = d1 && (__popc(m0) + __popc(m1 & lt) < avail);
    const unsigned k0 = __ballot_sync(0xffffffffu, d0), k1 = __ballot_sync(0xffffffffu, d1);
    if (lane == 0) {
        *q0 = k0;
        *q1 = k1;
        *cnt += __popc(k0) + __popc(k1);
    }
    __syncwarp();
}

// The accurate Newtonian pair (Newton-refined rsqrt) of the thread's two particles with one
// source staged as in acc_x2_j, plus its B side: c = -m_i r^-3 x_ji summed over the two
// particles, the deferred pairs left out (thrj: the source's threshold for this warp).
__device__ __forceinline__ void symdef_x2_j(const float4 A, const float4 B, const float4 C, const float2 M,
                                            float thrj, const AccX2I &P, const float2 nmi, float2 e2, int jglob,
                                            const float (&thr)[2], SmemSlots<2, SYM_BS> &big, float2 &ax,
                                            float2 &ay, float2 &az, float &cx, float &cy, float &cz, int *cnt,
                                            unsigned *q0, unsigned *q1, int lane)
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), P.nxh), __fadd2_rn(make_float2(B.z, B.w), P.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), P.nyh), __fadd2_rn(make_float2(C.x, C.y), P.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), P.nzh), __fadd2_rn(make_float2(C.z, C.w), P.nzl));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 nhy = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), r2), ri);
    ri = __ffma2_rn(ri, __ffma2_rn(nhy, ri, make_float2(0.5f, 0.5f)), ri);
    const float2 u = __fmul2_rn(ri, __fmul2_rn(ri, ri));  // r^-3
    float2 w = __fmul2_rn(M, u);                           // m_j r^-3
    float2 wj = __fmul2_rn(nmi, u);                        // -m_i r^-3
    if (__any_sync(0xffffffffu, (w.x > thr[0]) || (w.y > thr[1]))) {
        const bool b0 = (w.x > thr[0]) && big.room(0);
        if (b0) big.push(0, jglob);
        const bool b1 = (w.y > thr[1]) && big.room(1);
        if (b1) big.push(1, jglob);
        w.x = b0 ? 0.f : w.x;
        w.y = b1 ? 0.f : w.y;
    }
    ax = __ffma2_rn(w, dx, ax);
    ay = __ffma2_rn(w, dy, ay);
    az = __ffma2_rn(w, dz, az);
    bool d0 = wj.x < -thrj, d1 = wj.y < -thrj;
    bside_defer(d0, d1, cnt, q0, q1, lane);
    wj.x = d0 ? 0.f : wj.x;
    wj.y = d1 ? 0.f : wj.y;
    cx = fmaf(wj.y, dx.y, wj.x * dx.x);
    cy = fmaf(wj.y, dy.y, wj.x * dy.x);
    cz = fmaf(wj.y, dz.y, wj.x * dz.x);
}

// The gradient pair of the thread's two particles with one source staged as in grad_x2_j,
// plus its B side c = -m_i r^-3 (a_ji - 3 (x_ji . a_ji) x_ji / r^2) over the two particles.
__device__ __forceinline__ void gradsym_x2_j(const float4 G0, const float4 G1, const float4 G2, const float4 G3,
                                             const float4 G4, const float4 G5, const float4 G6, const float4 G7,
                                             float thrj, const GradX2I &P, const float2 nmi, float2 e2, int jglob,
                                             const float (&thr)[2], SmemSlots<2, SYM_BS> &big, float2 &gx,
                                             float2 &gy, float2 &gz, float &cx, float &cy, float &cz, int *cnt,
                                             unsigned *q0, unsigned *q1, int lane)
{
    const float2 dx = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(G0.x, G0.y), P.nxh),
                                            __fadd2_rn(make_float2(G1.z, G1.w), P.nxm)),
                                 __fadd2_rn(make_float2(G3.x, G3.y), P.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(G0.z, G0.w), P.nyh),
                                            __fadd2_rn(make_float2(G2.x, G2.y), P.nym)),
                                 __fadd2_rn(make_float2(G3.z, G3.w), P.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(G1.x, G1.y), P.nzh),
                                            __fadd2_rn(make_float2(G2.z, G2.w), P.nzm)),
                                 __fadd2_rn(make_float2(G4.x, G4.y), P.nzl));
    const float2 Ax = __fadd2_rn(__fadd2_rn(make_float2(G4.z, G4.w), P.nahx), __fadd2_rn(make_float2(G6.x, G6.y), P.nalx));
    const float2 Ay = __fadd2_rn(__fadd2_rn(make_float2(G5.x, G5.y), P.nahy), __fadd2_rn(make_float2(G6.z, G6.w), P.naly));
    const float2 Az = __fadd2_rn(__fadd2_rn(make_float2(G5.z, G5.w), P.nahz), __fadd2_rn(make_float2(G7.x, G7.y), P.nalz));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 nhy = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), r2), y);
    y = __ffma2_rn(y, __ffma2_rn(nhy, y, make_float2(0.5f, 0.5f)), y);
    const float2 ri2 = __fmul2_rn(y, y);
    const float2 u = __fmul2_rn(y, ri2);                             // r^-3
    float2 w = __fmul2_rn(make_float2(G7.z, G7.w), u);               // m_j r^-3
    float2 wj = __fmul2_rn(nmi, u);                                  // -m_i r^-3
    const bool b0 = (w.x > thr[0]) && big.room(0);
    if (b0) big.push(0, jglob);
    const bool b1 = (w.y > thr[1]) && big.room(1);
    if (b1) big.push(1, jglob);
    w.x = b0 ? 0.f : w.x;
    w.y = b1 ? 0.f : w.y;
    const float2 xa = __ffma2_rn(dx, Ax, __ffma2_rn(dy, Ay, __fmul2_rn(dz, Az)));
    const float2 nt3 = __fmul2_rn(__fmul2_rn(make_float2(-3.0f, -3.0f), xa), ri2);  // -3 (x.a) / r^2
    const float2 tx = __ffma2_rn(nt3, dx, Ax), ty = __ffma2_rn(nt3, dy, Ay), tz = __ffma2_rn(nt3, dz, Az);
    gx = __ffma2_rn(w, tx, gx);
    gy = __ffma2_rn(w, ty, gy);
    gz = __ffma2_rn(w, tz, gz);
    bool d0 = wj.x < -thrj, d1 = wj.y < -thrj;
    bside_defer(d0, d1, cnt, q0, q1, lane);
    wj.x = d0 ? 0.f : wj.x;
    wj.y = d1 ? 0.f : wj.y;
    cx = fmaf(wj.y, tx.y, wj.x * tx.x);
    cy = fmaf(wj.y, ty.y, wj.x * ty.x);
    cz = fmaf(wj.y, tz.y, wj.x * tz.x);
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS, 4) k_acc_sym_defer_mixed(const float4 *__restrict__ irec,
                                                            const float4 *__restrict__ jrec, int n_a, int n_s,
                                                            int nblk_i, int j_per_split, float eps2, double eps2d,
                                                            const float *__restrict__ wA,
                                                            const float *__restrict__ wB,
                                                            const int32_t *__restrict__ ilist,
                                                            const int32_t *__restrict__ jlist,
                                                            const double *__restrict__ mstore,
                                                            double *__restrict__ part, double *__restrict__ pj,
                                                            uint8_t *__restrict__ pcnt)
{
    constexpr int ILP = 2, W = BS / 32, FOLD = 16;
    static_assert(BS == SYM_BS && TJ == SYM_TJ, "slot columns and ballot rows are laid out for SYM_BS, SYM_TJ");
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ];
    __shared__ float2 sM[TJ];
    __shared__ float sT[W][TJ];
    __shared__ int sCnt[W][TJ];
    __shared__ float sJ[W][3][TJ];
    __shared__ unsigned sQ[W][ILP][TJ];
    __shared__ int s_slot[GRAD_SLOTS * ILP * BS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x, ng = gridDim.x;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    const float2 e2 = make_float2(eps2, eps2);
    const df::dfloat e2d = df::from_double(eps2d);
    for (int ib = g; ib < nblk_i; ib += ng) {
        const int ibase = ib * BS * ILP;
        // the thread's two particles; past the end: zero mass, far from every source
        float4 a0 = make_float4(SYM_FAR, SYM_FAR, SYM_FAR, 0.f), a1 = a0, b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
        const int i0 = ibase + tid, i1 = ibase + BS + tid;
        float thr[ILP] = {INFINITY, INFINITY};
        if (i0 < n_a) {
            a0 = irec[i0];
            b0 = irec[n_a + i0];
            thr[0] = SLOT_FRACTION * wA[i0];
        }
        if (i1 < n_a) {
            a1 = irec[i1];
            b1 = irec[n_a + i1];
            thr[1] = SLOT_FRACTION * wA[i1];
        }
        AccX2I P;
        P.nxh = make_float2(-a0.x, -a1.x);
        P.nyh = make_float2(-a0.y, -a1.y);
        P.nzh = make_float2(-a0.z, -a1.z);
        P.nxl = make_float2(-b0.x, -b1.x);
        P.nyl = make_float2(-b0.y, -b1.y);
        P.nzl = make_float2(-b0.z, -b1.z);
        const float2 nmi = make_float2(-a0.w, -a1.w);
        SmemSlots<ILP, BS> big;
        big.col = s_slot + tid;
        big.n[0] = big.n[1] = 0;
        float hx[ILP] = {0.f, 0.f}, hy[ILP] = {0.f, 0.f}, hz[ILP] = {0.f, 0.f};
        float lx[ILP] = {0.f, 0.f}, ly[ILP] = {0.f, 0.f}, lz[ILP] = {0.f, 0.f};
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            const int cnt8 = (cnt + 7) & ~7;
            __syncthreads();
            for (int t = tid; t < cnt8; t += BS) {
                float4 a = make_float4(-SYM_FAR, -SYM_FAR, -SYM_FAR, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
                float tj = INFINITY;
                if (t < cnt) {
                    a = jrec[j0 + t];
                    b = jrec[n_s + j0 + t];
                    tj = SLOT_FRACTION * wB[j0 + t];
                }
                sA[t] = make_float4(a.x, a.x, a.y, a.y);
                sB[t] = make_float4(a.z, a.z, b.x, b.x);
                sC[t] = make_float4(b.y, b.y, b.z, b.z);
                sM[t] = make_float2(a.w, a.w);
                stage_bside(sT, sCnt, sQ, pcnt, t, cnt, j0, n_s, g, ib == g, tj);
            }
            __syncthreads();
            for (int c0 = 0; c0 < cnt8; c0 += FOLD) {
                const int c1 = min(cnt8, c0 + FOLD);
                float2 ax2 = make_float2(0.f, 0.f), ay2 = ax2, az2 = ax2;
                // groups of 4 sources (a reduce-scatter of 8 would hold 12 more registers)
                for (int jj = c0; jj < c1; jj += 4) {
                    float cx[4], cy[4], cz[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int sj = jj + u;
                        symdef_x2_j(sA[sj], sB[sj], sC[sj], sM[sj], sT[warp][sj], P, nmi, e2, j0 + sj, thr, big, ax2,
                                    ay2, az2, cx[u], cy[u], cz[u], &sCnt[warp][sj], &sQ[warp][0][sj], &sQ[warp][1][sj],
                                    lane);
                    }
                    const float rx = reduce_scatter4(cx, lane);
                    const float ry = reduce_scatter4(cy, lane);
                    const float rz = reduce_scatter4(cz, lane);
                    if ((lane & 7) == 0) {
                        const int s = jj + (lane >> 3);
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
            // the tile's B side: the FP32 sums over the block's particles, then the deferred
            // terms in double-float in a fixed order, added to the group's partials
            for (int t = tid; t < cnt; t += BS) {
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v = sJ[0][c][t];
#pragma unroll
                    for (int q = 1; q < W; ++q) v += sJ[q][c][t];
                    d[c] = (double)v;
                }
                const int j = j0 + t;
                unsigned anyq = 0u;
#pragma unroll
                for (int q = 0; q < W; ++q) anyq |= sQ[q][0][t] | sQ[q][1][t];
                if (anyq) {
                    const float4 ja = jrec[j], jl = jrec[n_s + j];
                    DF3 b = df3_zero();
                    double f[3] = {0.0, 0.0, 0.0};
                    for (int q = 0; q < W; ++q)
                        for (int k = 0; k < ILP; ++k) {
                            unsigned mk = sQ[q][k][t];
                            while (mk) {
                                const int i = ibase + k * BS + q * 32 + (__ffs(mk) - 1);
                                mk &= mk - 1u;
                                const float4 I0 = irec[i], I1 = irec[n_a + i];
                                DF3 r;
                                if (acc_term_df3(I0, I1, ja.x, ja.y, ja.z, jl.x, jl.y, jl.z, e2d, r)) {
                                    df3_add(b, r);
                                } else {
                                    const D3 u = acc_term_fp64(I0, I1, ja.x, ja.y, ja.z, jl.x, jl.y, jl.z,
                                                               mstore[ilist ? ilist[i] : i], eps2d);
                                    f[0] += u.x;
                                    f[1] += u.y;
                                    f[2] += u.z;
                                }
                            }
                        }
                    d[0] += df::to_double(b.x) + f[0];
                    d[1] += df::to_double(b.y) + f[1];
                    d[2] += df::to_double(b.z) + f[2];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double *dst = pj + ((size_t)g * 3 + c) * n_s + j;
                    *dst = (ib == g) ? d[c] : *dst + d[c];
                }
#pragma unroll
                for (int w = 0; w < W; ++w) pcnt[((size_t)g * W + w) * n_s + j] = (uint8_t)sCnt[w][t];
            }
        }
        // the A side of this i-block and split: the FP32 sums, then the deferred terms
        double res[ILP][3];
        res[0][0] = (double)hx[0] + (double)lx[0];
        res[0][1] = (double)hy[0] + (double)ly[0];
        res[0][2] = (double)hz[0] + (double)lz[0];
        res[1][0] = (double)hx[1] + (double)lx[1];
        res[1][1] = (double)hy[1] + (double)ly[1];
        res[1][2] = (double)hz[1] + (double)lz[1];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const float4 ia = k ? a1 : a0, il = k ? b1 : b0;
            DF3 b = df3_zero();
            double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int s = 0; s < GRAD_SLOTS; ++s) {
                if (s < big.n[k]) {
                    const int j = big.get(s, k);
                    const float4 J0 = jrec[j], J1 = jrec[n_s + j];
                    DF3 t;
                    if (acc_term_df3(J0, J1, ia.x, ia.y, ia.z, il.x, il.y, il.z, e2d, t)) {
                        df3_add(b, t);
                    } else {
                        const D3 u = acc_term_fp64(J0, J1, ia.x, ia.y, ia.z, il.x, il.y, il.z,
                                                   mstore[jlist ? jlist[j] : j], eps2d);
                        f[0] += u.x;
                        f[1] += u.y;
                        f[2] += u.z;
                    }
                }
            }
            res[k][0] += df::to_double(b.x) + f[0];
            res[k][1] += df::to_double(b.y) + f[1];
            res[k][2] += df::to_double(b.z) + f[2];
        }
        double *p = part + (size_t)blockIdx.y * 3 * n_a;
        if (i0 < n_a) {
            p[i0] = res[0][0];
            p[n_a + i0] = res[0][1];
            p[2 * n_a + i0] = res[0][2];
        }
        if (i1 < n_a) {
            p[i1] = res[1][0];
            p[n_a + i1] = res[1][1];
            p[2 * n_a + i1] = res[1][2];
        }
    }
}

// one particle's gradient record (the four float4 of launch_pack_grad_mixed) as GradMixedI<1>
__device__ __forceinline__ GradMixedI<1> grad_rec_of(const float4 *__restrict__ rec, int n, int i)
{
    const float4 q0 = rec[i], q1 = rec[n + i], q2 = rec[2 * n + i], q3 = rec[3 * n + i];
    GradMixedI<1> O;
    O.xh[0] = q0.x; O.yh[0] = q0.y; O.zh[0] = q0.z;
    O.xm[0] = q1.x; O.ym[0] = q1.y; O.zm[0] = q1.z; O.ahx[0] = q1.w;
    O.xl[0] = q2.x; O.yl[0] = q2.y; O.zl[0] = q2.z; O.ahy[0] = q2.w;
    O.ahz[0] = q3.x; O.alx[0] = q3.y; O.aly[0] = q3.z; O.alz[0] = q3.w;
    return O;
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS, 4) k_grad_sym_mixed(const float4 *__restrict__ irec,
                                                       const float4 *__restrict__ jrec, int n_a, int n_s, int nblk_i,
                                                       int j_per_split, double eps2d, const float *__restrict__ wA,
                                                       const float *__restrict__ wB, double *__restrict__ part,
                                                       double *__restrict__ pj, uint8_t *__restrict__ pcnt)
{
    constexpr int ILP = 2, W = BS / 32, FOLD = 64;
    static_assert(BS == SYM_BS && TJ == SYM_TJ, "slot columns and ballot rows are laid out for SYM_BS, SYM_TJ");
    __shared__ float4 sG[8][TJ];
    __shared__ float sT[W][TJ];
    __shared__ int sCnt[W][TJ];
    __shared__ float sJ[W][3][TJ];
    __shared__ unsigned sQ[W][ILP][TJ];
    __shared__ int s_slot[GRAD_SLOTS * ILP * BS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x, ng = gridDim.x;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    const float eps2 = (float)eps2d;
    const float2 e2 = make_float2(eps2, eps2);
    const df::dfloat e2d = df::from_double(eps2d);
    for (int ib = g; ib < nblk_i; ib += ng) {
        const int ibase = ib * BS * ILP;
        const int i0 = ibase + tid, i1 = ibase + BS + tid;
        // the thread's two particles; past the end: zero mass, far from every source
        float4 q[ILP][4];
        float thr[ILP] = {INFINITY, INFINITY};
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const int i = k ? i1 : i0;
            q[k][0] = make_float4(SYM_FAR, SYM_FAR, SYM_FAR, 0.f);
            q[k][1] = q[k][2] = q[k][3] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n_a) {
                q[k][0] = irec[i];
                q[k][1] = irec[n_a + i];
                q[k][2] = irec[2 * n_a + i];
                q[k][3] = irec[3 * n_a + i];
                thr[k] = SLOT_FRACTION * wA[i];
            }
        }
        GradX2I P;
        P.nxh = make_float2(-q[0][0].x, -q[1][0].x);
        P.nyh = make_float2(-q[0][0].y, -q[1][0].y);
        P.nzh = make_float2(-q[0][0].z, -q[1][0].z);
        P.nxm = make_float2(-q[0][1].x, -q[1][1].x);
        P.nym = make_float2(-q[0][1].y, -q[1][1].y);
        P.nzm = make_float2(-q[0][1].z, -q[1][1].z);
        P.nxl = make_float2(-q[0][2].x, -q[1][2].x);
        P.nyl = make_float2(-q[0][2].y, -q[1][2].y);
        P.nzl = make_float2(-q[0][2].z, -q[1][2].z);
        P.nahx = make_float2(-q[0][1].w, -q[1][1].w);
        P.nahy = make_float2(-q[0][2].w, -q[1][2].w);
        P.nahz = make_float2(-q[0][3].x, -q[1][3].x);
        P.nalx = make_float2(-q[0][3].y, -q[1][3].y);
        P.naly = make_float2(-q[0][3].z, -q[1][3].z);
        P.nalz = make_float2(-q[0][3].w, -q[1][3].w);
        const float2 nmi = make_float2(-q[0][0].w, -q[1][0].w);
        SmemSlots<ILP, BS> big;
        big.col = s_slot + tid;
        big.n[0] = big.n[1] = 0;
        float hx[ILP] = {0.f, 0.f}, hy[ILP] = {0.f, 0.f}, hz[ILP] = {0.f, 0.f};
        float lx[ILP] = {0.f, 0.f}, ly[ILP] = {0.f, 0.f}, lz[ILP] = {0.f, 0.f};
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            const int cnt8 = (cnt + 7) & ~7;
            __syncthreads();
            for (int t = tid; t < cnt8; t += BS) {
                float4 r0 = make_float4(-SYM_FAR, -SYM_FAR, -SYM_FAR, 0.f), r1 = make_float4(0.f, 0.f, 0.f, 0.f),
                       r2 = r1, r3 = r1;
                float tj = INFINITY;
                if (t < cnt) {
                    r0 = jrec[j0 + t];
                    r1 = jrec[n_s + j0 + t];
                    r2 = jrec[2 * n_s + j0 + t];
                    r3 = jrec[3 * n_s + j0 + t];
                    tj = SLOT_FRACTION * wB[j0 + t];
                }
                sG[0][t] = make_float4(r0.x, r0.x, r0.y, r0.y);
                sG[1][t] = make_float4(r0.z, r0.z, r1.x, r1.x);
                sG[2][t] = make_float4(r1.y, r1.y, r1.z, r1.z);
                sG[3][t] = make_float4(r2.x, r2.x, r2.y, r2.y);
                sG[4][t] = make_float4(r2.z, r2.z, r1.w, r1.w);
                sG[5][t] = make_float4(r2.w, r2.w, r3.x, r3.x);
                sG[6][t] = make_float4(r3.y, r3.y, r3.z, r3.z);
                sG[7][t] = make_float4(r3.w, r3.w, r0.w, r0.w);
                stage_bside(sT, sCnt, sQ, pcnt, t, cnt, j0, n_s, g, ib == g, tj);
            }
            __syncthreads();
            for (int c0 = 0; c0 < cnt8; c0 += FOLD) {
                const int c1 = min(cnt8, c0 + FOLD);
                float2 gx2 = make_float2(0.f, 0.f), gy2 = gx2, gz2 = gx2;
                // groups of 4 sources (a reduce-scatter of 8 would hold 12 more registers)
                for (int jj = c0; jj < c1; jj += 4) {
                    float cx[4], cy[4], cz[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int s = jj + u;
                        gradsym_x2_j(sG[0][s], sG[1][s], sG[2][s], sG[3][s], sG[4][s], sG[5][s], sG[6][s], sG[7][s],
                                     sT[warp][s], P, nmi, e2, j0 + s, thr, big, gx2, gy2, gz2, cx[u], cy[u], cz[u],
                                     &sCnt[warp][s], &sQ[warp][0][s], &sQ[warp][1][s], lane);
                    }
                    const float rx = reduce_scatter4(cx, lane);
                    const float ry = reduce_scatter4(cy, lane);
                    const float rz = reduce_scatter4(cz, lane);
                    if ((lane & 7) == 0) {
                        const int s = jj + (lane >> 3);
                        sJ[warp][0][s] = rx;
                        sJ[warp][1][s] = ry;
                        sJ[warp][2][s] = rz;
                    }
                }
                fold2(hx[0], lx[0], gx2.x);
                fold2(hy[0], ly[0], gy2.x);
                fold2(hz[0], lz[0], gz2.x);
                fold2(hx[1], lx[1], gx2.y);
                fold2(hy[1], ly[1], gy2.y);
                fold2(hz[1], lz[1], gz2.y);
            }
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v = sJ[0][c][t];
#pragma unroll
                    for (int w = 1; w < W; ++w) v += sJ[w][c][t];
                    d[c] = (double)v;
                }
                const int j = j0 + t;
                unsigned anyq = 0u;
#pragma unroll
                for (int w = 0; w < W; ++w) anyq |= sQ[w][0][t] | sQ[w][1][t];
                if (anyq) {
                    const GradMixedI<1> O = grad_rec_of(jrec, n_s, j);
                    DF3 b = df3_zero();
                    double f[3] = {0.0, 0.0, 0.0};
                    for (int w = 0; w < W; ++w)
                        for (int k = 0; k < ILP; ++k) {
                            unsigned mk = sQ[w][k][t];
                            while (mk) {
                                const int i = ibase + k * BS + w * 32 + (__ffs(mk) - 1);
                                mk &= mk - 1u;
                                const float4 I0 = irec[i], I1 = irec[n_a + i], I2 = irec[2 * n_a + i],
                                             I3 = irec[3 * n_a + i];
                                DF3 r;
                                if (grad_term_df3<1>(I0, I1, I2, I3, O, 0, e2d, r)) df3_add(b, r);
                                else grad_term_fp64<1>(I0, I1, I2, I3, O, 0, eps2d, f[0], f[1], f[2]);
                            }
                        }
                    d[0] += df::to_double(b.x) + f[0];
                    d[1] += df::to_double(b.y) + f[1];
                    d[2] += df::to_double(b.z) + f[2];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double *dst = pj + ((size_t)g * 3 + c) * n_s + j;
                    *dst = (ib == g) ? d[c] : *dst + d[c];
                }
#pragma unroll
                for (int w = 0; w < W; ++w) pcnt[((size_t)g * W + w) * n_s + j] = (uint8_t)sCnt[w][t];
            }
        }
        double *p = part + (size_t)blockIdx.y * 3 * n_a;
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const int i = k ? i1 : i0;
            double bx = 0.0, by = 0.0, bz = 0.0;
            if (big.n[k] > 0) {
                const GradMixedI<1> O = grad_rec_of(irec, n_a, i);
                DF3 b = df3_zero();
                for (int s = 0; s < big.n[k]; ++s) {
                    const int j = big.get(s, k);
                    const float4 J0 = jrec[j], J1 = jrec[n_s + j], J2 = jrec[2 * n_s + j], J3 = jrec[3 * n_s + j];
                    DF3 t;
                    if (grad_term_df3<1>(J0, J1, J2, J3, O, 0, e2d, t)) df3_add(b, t);
                    else grad_term_fp64<1>(J0, J1, J2, J3, O, 0, eps2d, bx, by, bz);
                }
                bx += df::to_double(b.x);
                by += df::to_double(b.y);
                bz += df::to_double(b.z);
            }
            if (i < n_a) {
                p[i] = ((double)hx[k] + (double)lx[k]) + bx;
                p[n_a + i] = ((double)hy[k] + (double)ly[k]) + by;
                p[2 * n_a + i] = ((double)hz[k] + (double)lz[k]) + bz;
            }
        }
    }
}

}  // namespace

void launch_acc_sym_defer(cudaStream_t s, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                          const float *wA, const float *wB, const int32_t *ilist, const int32_t *jlist,
                          const double *mstore, double *part, double *pj, uint8_t *pcnt, const SymShape &sh)
{
    const dim3 grid(sh.ngroups, sh.nsplit);
    k_acc_sym_defer_mixed<SYM_BS, SYM_TJ><<<grid, SYM_BS, 0, s>>>((const float4 *)irec, (const float4 *)jrec, n_a,
                                                                  n_s, sh.nblk_i, sh.j_per_split, (float)eps2, eps2,
                                                                  wA, wB, ilist, jlist, mstore, part, pj, pcnt);
}

void launch_grad_sym(cudaStream_t s, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                     const float *wA, const float *wB, double *part, double *pj, uint8_t *pcnt, const SymShape &sh)
{
    const dim3 grid(sh.ngroups, sh.nsplit);
    k_grad_sym_mixed<SYM_BS, SYM_TJ><<<grid, SYM_BS, 0, s>>>((const float4 *)irec, (const float4 *)jrec, n_a, n_s,
                                                             sh.nblk_i, sh.j_per_split, eps2, wA, wB, part, pj, pcnt);
}

}  // namespace frost
