// Integrator and bookkeeping kernels of the HHS-FSI hot path for sm_103a:
//   kick / drift (Sec. 5.3), the stable slow/fast partition (Sec. 3.1), index-list
//   validation, and the FP64 energy / momentum / angular-momentum reductions (Sec. 2.3).
#include "df_arith.cuh"
#include "frost_internal.cuh"
#include "pair_bodies.cuh"

#include <cmath>

namespace frost {
namespace {

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__global__ void k_kick(const int32_t *__restrict__ list, int n, double *__restrict__ v, int N,
                       const double *__restrict__ a, double dt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list ? list[k] : k;
    // separate roundings of the product and the sum (no contraction into an FMA)
    v[i] = __dadd_rn(v[i], __dmul_rn(dt, a[k]));
    v[N + i] = __dadd_rn(v[N + i], __dmul_rn(dt, a[n + k]));
    v[2 * N + i] = __dadd_rn(v[2 * N + i], __dmul_rn(dt, a[2 * n + k]));
}

__global__ void k_kick_by_particle(const int32_t *__restrict__ list, int n, double *__restrict__ v, int N,
                                   const double *__restrict__ a, double dt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list ? list[k] : k;
    v[i] = __dadd_rn(v[i], __dmul_rn(dt, a[i]));
    v[N + i] = __dadd_rn(v[N + i], __dmul_rn(dt, a[N + i]));
    v[2 * N + i] = __dadd_rn(v[2 * N + i], __dmul_rn(dt, a[2 * N + i]));
}

__global__ void k_kick_aos(const int32_t *__restrict__ list, int n, double *__restrict__ v, int N,
                           const double *__restrict__ a, double dt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list ? list[k] : k;
    v[i] = __dadd_rn(v[i], __dmul_rn(dt, a[3 * k]));
    v[N + i] = __dadd_rn(v[N + i], __dmul_rn(dt, a[3 * k + 1]));
    v[2 * N + i] = __dadd_rn(v[2 * N + i], __dmul_rn(dt, a[3 * k + 2]));
}

__global__ void k_drift(const int32_t *__restrict__ list, int n, double *__restrict__ x,
                        const double *__restrict__ v, int N, double dt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list ? list[k] : k;
    x[i] = __dadd_rn(x[i], __dmul_rn(dt, v[i]));
    x[N + i] = __dadd_rn(x[N + i], __dmul_rn(dt, v[N + i]));
    x[2 * N + i] = __dadd_rn(x[2 * N + i], __dmul_rn(dt, v[2 * N + i]));
}

// drift, then the position record of the moved particle for the next Newtonian pass
__global__ void k_drift_pack(const int32_t *__restrict__ list, int n, double *__restrict__ x,
                             const double *__restrict__ v, const double *__restrict__ m, int N, double dt,
                             void *__restrict__ rec, int mode)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list ? list[k] : k;
    x[i] = __dadd_rn(x[i], __dmul_rn(dt, v[i]));
    x[N + i] = __dadd_rn(x[N + i], __dmul_rn(dt, v[N + i]));
    x[2 * N + i] = __dadd_rn(x[2 * N + i], __dmul_rn(dt, v[2 * N + i]));
    if (mode == 0) dev::pack_pos_mixed_one(k, list, n, x, m, N, (float4 *)rec);
    else dev::pack_pos_fp64_one(k, list, n, x, m, N, (double4_32a *)rec);
}

// Stable partition by one block of 1024 threads: chunks of 1024 entries, slow ranks from a
// warp-ballot prefix count, fast ranks as the complement.
__global__ void __launch_bounds__(1024) k_partition(const int32_t *__restrict__ set, int n,
                                                    const double *__restrict__ tau, double pivot,
                                                    int32_t *__restrict__ S, int32_t *__restrict__ F,
                                                    int64_t *__restrict__ counts)
{
    __shared__ int wsum[32];
    __shared__ int chunk_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int sbase = 0, fbase = 0;
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int k = c0 + tid;
        const bool valid = k < n;
        const bool slow = valid && (tau[k] >= pivot);
        const unsigned bal = __ballot_sync(0xffffffffu, slow);
        const int rank = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int vsum = wsum[lane];
            int incl = vsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            wsum[lane] = incl - vsum;  // exclusive prefix of slow counts per warp
            if (lane == 31) chunk_total = incl;
        }
        __syncthreads();
        if (valid) {
            const int sidx = wsum[warp] + rank;  // slow entries before k in this chunk
            const int id = set ? set[k] : k;
            if (slow) S[sbase + sidx] = id;
            else F[fbase + (tid - sidx)] = id;
        }
        const int tot = chunk_total;
        const int nvalid = min(1024, n - c0);
        sbase += tot;
        fbase += nvalid - tot;
        __syncthreads();
    }
    if (tid == 0) {
        counts[0] = sbase;
        counts[1] = fbase;
    }
}

// The same stable partition by many blocks, for large sets: block b takes the entries
// [b PART_CHUNK, (b + 1) PART_CHUNK).  k_part_count writes each block's slow count; k_part_scatter
// starts each block at the slow and fast counts of the blocks before it and compacts its entries
// with the single-block kernel's ballot scan, so S and F are the same lists in the same order.
constexpr int PART_CHUNK = 4096;

__device__ __forceinline__ int block_sum_1024(int c, int *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __syncthreads();  // wsum may still be read from an earlier use
    if (lane == 0) wsum[warp] = c;
    __syncthreads();
    int t = 0;
    for (int q = 0; q < 32; ++q) t += wsum[q];
    return t;
}

__global__ void __launch_bounds__(1024) k_part_count(int n, const double *__restrict__ tau, double pivot,
                                                     int *__restrict__ blk)
{
    __shared__ int wsum[32];
    const int lo = blockIdx.x * PART_CHUNK, hi = min(n, lo + PART_CHUNK);
    int c = 0;
    for (int k = lo + threadIdx.x; k < hi; k += 1024) c += (tau[k] >= pivot) ? 1 : 0;
    const int t = block_sum_1024(c, wsum);
    if (threadIdx.x == 0) blk[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_part_scatter(const int32_t *__restrict__ set, int n,
                                                       const double *__restrict__ tau, double pivot,
                                                       const int *__restrict__ blk, int32_t *__restrict__ S,
                                                       int32_t *__restrict__ F, int64_t *__restrict__ counts)
{
    __shared__ int wsum[32];
    __shared__ int chunk_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lo = blockIdx.x * PART_CHUNK, hi = min(n, lo + PART_CHUNK);
    int before = 0;
    for (int b = tid; b < (int)blockIdx.x; b += 1024) before += blk[b];
    int sbase = block_sum_1024(before, wsum);
    int fbase = lo - sbase;
    for (int c0 = lo; c0 < hi; c0 += 1024) {
        const int k = c0 + tid;
        const bool valid = k < hi;
        const bool slow = valid && (tau[k] >= pivot);
        const unsigned bal = __ballot_sync(0xffffffffu, slow);
        const int rank = __popc(bal & ((1u << lane) - 1u));
        __syncthreads();  // every thread has read wsum (block sum or the previous chunk)
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int vsum = wsum[lane];
            int incl = vsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            wsum[lane] = incl - vsum;  // exclusive prefix of slow counts per warp
            if (lane == 31) chunk_total = incl;
        }
        __syncthreads();
        if (valid) {
            const int sidx = wsum[warp] + rank;  // slow entries before k in this chunk
            const int id = set ? set[k] : k;
            if (slow) S[sbase + sidx] = id;
            else F[fbase + (tid - sidx)] = id;
        }
        const int tot = chunk_total;
        const int nvalid = min(1024, hi - c0);
        sbase += tot;
        fbase += nvalid - tot;
    }
    if (tid == 0 && blockIdx.x == gridDim.x - 1) {
        counts[0] = sbase;
        counts[1] = fbase;
    }
}

// list relation: B adds 1 to its marks, A adds 2; a repeated entry sees its own bit already set
__global__ void k_mark_B(const int32_t *__restrict__ B, int nB, int N, int32_t *__restrict__ marks,
                         int64_t *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nB) return;
    const int i = B ? B[k] : k;
    if (i < 0 || i >= N) {
        out[0] = 1;
        return;
    }
    if (atomicAdd(&marks[i], 1) & 1) out[0] = 1;
}

__global__ void k_mark_A(const int32_t *__restrict__ A, int nA, int N, int32_t *__restrict__ marks,
                         int64_t *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nA) return;
    const int i = A ? A[k] : k;
    if (i < 0 || i >= N) {
        out[0] = 1;
        return;
    }
    const int old = atomicAdd(&marks[i], 2);
    if (old & 2) out[0] = 1;
    if (old & 1) atomicAdd((unsigned long long *)&out[1], 1ull);
}

__global__ void k_unmark(const int32_t *__restrict__ L, int n, int N, int32_t *__restrict__ marks)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = L ? L[k] : k;
    if (i >= 0 && i < N) marks[i] = 0;
}

__global__ void k_check_finite(const double *__restrict__ p, int64_t n, int *__restrict__ err)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(p[k])) atomicOr(err, ERR_NONFINITE);
}

__global__ void k_identity(int32_t *__restrict__ list, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) list[k] = k;
}

// [n][3] <-> [3][n] layout conversion of a particle vector
__global__ void k_aos_to_soa(const double *__restrict__ aos, int n, double *__restrict__ soa,
                             int *__restrict__ err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    bool ok = true;
    for (int c = 0; c < 3; ++c) {
        const double q = aos[3 * (size_t)k + c];
        ok = ok && isfinite(q);
        soa[(size_t)c * n + k] = q;
    }
    if (!ok) atomicOr(err, ERR_NONFINITE);
}

__global__ void k_soa_to_aos(const double *__restrict__ soa, int n, double *__restrict__ aos)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    for (int c = 0; c < 3; ++c) aos[3 * (size_t)k + c] = soa[(size_t)c * n + k];
}

// masses must be finite and positive
__global__ void k_check_mass(const double *__restrict__ m, int n, int *__restrict__ err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (!(m[k] > 0.0) || !isfinite(m[k])) atomicOr(err, ERR_NONFINITE);
}

// ---- potential in double-float arithmetic (df_arith.cuh) ---------------------------------
// The O(N^2) potential of the energy diagnostic runs on the FP32 pipes and keeps about 1e-13
// relative accuracy per phi_i (positions enter exactly, as three FP32 parts).

// records: p0 = {x_h, y_h, z_h, m_h}, p1 = {x_l, y_l, z_l, m_l}, p2 = {x_ll, y_ll, z_ll, 0}
__global__ void k_pack_pot_df(const double *__restrict__ x, const double *__restrict__ m, int N,
                              float4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float xh, xl, xll, yh, yl, yll, zh, zl, zll;
    df::split3(x[i], xh, xl, xll);
    df::split3(x[N + i], yh, yl, yll);
    df::split3(x[2 * N + i], zh, zl, zll);
    const double pm = m[i];
    const float hm = (float)pm;
    rec[i] = make_float4(xh, yh, zh, hm);
    rec[N + i] = make_float4(xl, yl, zl, (float)(pm - (double)hm));
    rec[2 * N + i] = make_float4(xll, yll, zll, 0.f);
}


// phi_i = sum_{j > i} m_j / sqrt(r^2 + eps2) in double-float, j-split partials part[split][i]:
// each pair once (U = -G sum_i m_i phi_i); the tiles wholly at or below the block's i-range are
// skipped, so the pass does half the pairs of the full sum
template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_potential_df(const float4 *__restrict__ rec, int n,
                                                     int j_per_split, double eps2,
                                                     double *__restrict__ part)
{
    __shared__ float4 s0[TJ], s1[TJ], s2[TJ];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * BS + tid;
    float4 I0 = make_float4(0.f, 0.f, 0.f, 0.f), I1 = I0, I2 = I0;
    if (i < n) {
        I0 = rec[i];
        I1 = rec[n + i];
        I2 = rec[2 * n + i];
    }
    const float e2h = (float)eps2, e2l = (float)(eps2 - (double)e2h);
    float H = 0.f, L = 0.f;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n, jb + j_per_split);
    const int ibase = blockIdx.x * BS;
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        if (j0 + cnt <= ibase + 1) continue;  // no j > i in this tile (block-uniform)
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            s0[t] = rec[j0 + t];
            s1[t] = rec[n + j0 + t];
            s2[t] = rec[2 * n + j0 + t];
        }
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 J0 = s0[jj], J1 = s1[jj], J2 = s2[jj];
            const df::dfloat sx = df::sep(J0.x, J1.x, J2.x, I0.x, I1.x, I2.x);
            const df::dfloat sy = df::sep(J0.y, J1.y, J2.y, I0.y, I1.y, I2.y);
            const df::dfloat sz = df::sep(J0.z, J1.z, J2.z, I0.z, I1.z, I2.z);
            const float xh = sx.h, xl = sx.l, yh = sy.h, yl = sy.l, zh = sz.h, zl = sz.l;
            // r^2 + eps^2: exact squares of the high parts, first-order terms of the low parts
            // (products feeding an error-free transformation are rounded on their own, __fmul_rn,
            // so that the compiler cannot contract them into the following add)
            const float px = __fmul_rn(xh, xh), py = __fmul_rn(yh, yh), pz = __fmul_rn(zh, zh);
            const float qx = fmaf(xh + xh, xl, fmaf(xh, xh, -px));
            const float qy = fmaf(yh + yh, yl, fmaf(yh, yh, -py));
            const float qz = fmaf(zh + zh, zl, fmaf(zh, zh, -pz));
            float s, t, S, u, S2, u2;
            df::two_sum(px, py, s, t);
            df::two_sum(s, pz, S, u);
            df::two_sum(S, e2h, S2, u2);
            const float lo = ((t + u) + (u2 + e2l)) + ((qx + qy) + qz);
            // 1 / r: MUFU estimate y0 and the residual res = 1 - r^2 y0^2 in double-float; then
            // 1/r = y0 (1 - res)^(-1/2) = y0 (1 + res/2 + 3 res^2/8 + ...), |res| < 2^-21
            const float y0 = rsqrtf(S2);
            const float q = __fmul_rn(y0, y0), qe = fmaf(y0, y0, -q);
            const float pp = __fmul_rn(S2, q), pe = fmaf(S2, q, -pp);
            const float res = ((1.f - pp) - pe) - fmaf(S2, qe, lo * q);
            const float c = y0 * res * fmaf(0.375f, res, 0.5f);
            // m_j / r = (m_h + m_l)(y0 + c)
            const float w = __fmul_rn(J0.w, y0);
            const float we = fmaf(J0.w, y0, -w) + fmaf(J0.w, c, J1.w * y0);
            if (j0 + jj > i) {
                float e;
                df::two_sum(H, w, H, e);
                L += e + we;
            }
        }
    }
    if (i < n) part[(size_t)blockIdx.y * n + i] = (double)H + (double)L;
}

// Per-cluster FP64 energy, momentum and angular momentum: block b reduces cluster
// [offsets[b], offsets[b+1]) in a fixed order.  out[b][8] = {T, sum_{i<j} m_i m_j / r, P, L}.
__global__ void __launch_bounds__(256) k_cluster_energy(const int64_t *__restrict__ offsets,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ v,
                                                        const double *__restrict__ m, int N,
                                                        double eps2, double *__restrict__ out)
{
    __shared__ double red[8][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lo = (int)offsets[blockIdx.x], hi = (int)offsets[blockIdx.x + 1];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = lo + tid; i < hi; i += 256) {
        const double mi = m[i];
        const double px = x[i], py = x[N + i], pz = x[2 * N + i];
        const double ux = v[i], uy = v[N + i], uz = v[2 * N + i];
        double phi = 0.0;
        for (int j = i + 1; j < hi; ++j) {
            const double dx = x[j] - px, dy = x[N + j] - py, dz = x[2 * N + j] - pz;
            phi += m[j] * rsqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2))));
        }
        acc[0] += 0.5 * mi * (ux * ux + uy * uy + uz * uz);
        acc[1] += mi * phi;
        acc[2] += mi * ux;
        acc[3] += mi * uy;
        acc[4] += mi * uz;
        acc[5] += mi * (py * uz - pz * uy);
        acc[6] += mi * (pz * ux - px * uz);
        acc[7] += mi * (px * uy - py * ux);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double a = acc[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (tid < 8) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w) a += red[tid][w];
        out[(size_t)blockIdx.x * 8 + tid] = a;
    }
}

// Single-block FP64 reduction in a fixed order (deterministic).
__global__ void __launch_bounds__(1024) k_energy_reduce(const double *__restrict__ x,
                                                        const double *__restrict__ v,
                                                        const double *__restrict__ m, int N,
                                                        const double *__restrict__ part, int nsplit,
                                                        double *__restrict__ out)
{
    __shared__ double red[8][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = tid; i < N; i += 1024) {
        const double mi = m[i];
        const double px = x[i], py = x[N + i], pz = x[2 * N + i];
        const double ux = v[i], uy = v[N + i], uz = v[2 * N + i];
        double phi = 0.0;
        for (int p = 0; p < nsplit; ++p) phi += part[(size_t)p * N + i];
        acc[0] += 0.5 * mi * (ux * ux + uy * uy + uz * uz);
        acc[1] += mi * phi;
        acc[2] += mi * ux;
        acc[3] += mi * uy;
        acc[4] += mi * uz;
        acc[5] += mi * (py * uz - pz * uy);
        acc[6] += mi * (pz * ux - px * uz);
        acc[7] += mi * (px * uy - py * ux);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double a = acc[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double a = red[q][lane];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) out[q] = a;
        }
    }
}

}  // namespace

void launch_kick(cudaStream_t s, const int32_t *list, int n, double *v, int N, const double *a_soa,
                 double dt)
{
    if (n <= 0) return;
    k_kick<<<cdiv(n, 256), 256, 0, s>>>(list, n, v, N, a_soa, dt);
}

void launch_kick_by_particle(cudaStream_t s, const int32_t *list, int n, double *v, int N,
                             const double *a_glob, double dt)
{
    if (n <= 0) return;
    k_kick_by_particle<<<cdiv(n, 256), 256, 0, s>>>(list, n, v, N, a_glob, dt);
}

void launch_kick_aos(cudaStream_t s, const int32_t *list, int n, double *v, int N,
                     const double *a_aos, double dt)
{
    if (n <= 0) return;
    k_kick_aos<<<cdiv(n, 256), 256, 0, s>>>(list, n, v, N, a_aos, dt);
}

void launch_drift(cudaStream_t s, const int32_t *list, int n, double *x, const double *v, int N,
                  double dt)
{
    if (n <= 0) return;
    k_drift<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, v, N, dt);
}

void launch_drift_pack(cudaStream_t s, const int32_t *list, int n, double *x, const double *v,
                       const double *m, int N, double dt, void *rec, int mode)
{
    if (n <= 0) return;
    k_drift_pack<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, v, m, N, dt, rec, mode);
}

void launch_partition(cudaStream_t s, const int32_t *set, int n, const double *tau, double pivot,
                      int32_t *S, int32_t *F, int64_t *counts, int *blk)
{
    if (blk && n >= PART_MULTI_MIN) {
        const int nb = cdiv(n, PART_CHUNK);
        k_part_count<<<nb, 1024, 0, s>>>(n, tau, pivot, blk);
        k_part_scatter<<<nb, 1024, 0, s>>>(set, n, tau, pivot, blk, S, F, counts);
        return;
    }
    k_partition<<<1, 1024, 0, s>>>(set, n, tau, pivot, S, F, counts);
}

void launch_list_relation(cudaStream_t s, const int32_t *A, int nA, const int32_t *B, int nB,
                          int N, int32_t *marks, int64_t *out)
{
    cudaMemsetAsync(out, 0, 2 * sizeof(int64_t), s);
    if (nB > 0) k_mark_B<<<cdiv(nB, 256), 256, 0, s>>>(B, nB, N, marks, out);
    if (nA > 0) k_mark_A<<<cdiv(nA, 256), 256, 0, s>>>(A, nA, N, marks, out);
    if (nB > 0) k_unmark<<<cdiv(nB, 256), 256, 0, s>>>(B, nB, N, marks);
    if (nA > 0) k_unmark<<<cdiv(nA, 256), 256, 0, s>>>(A, nA, N, marks);
}

void launch_check_finite(cudaStream_t s, const double *p, int64_t n, int *err)
{
    if (n <= 0) return;
    const unsigned nb = (unsigned)std::min<long long>(4096, (n + 255) / 256);
    k_check_finite<<<nb, 256, 0, s>>>(p, n, err);
}

void launch_identity(cudaStream_t s, int32_t *list, int n)
{
    if (n <= 0) return;
    k_identity<<<cdiv(n, 256), 256, 0, s>>>(list, n);
}

void launch_potential(cudaStream_t s, const double *x, const double *m, int n, double eps2, float4 *rec,
                      double *part, const SplitShape &shape)
{
    if (n <= 0) return;
    k_pack_pot_df<<<cdiv(n, 256), 256, 0, s>>>(x, m, n, rec);
    const dim3 grid(shape.nblk_i, shape.nsplit);
    k_potential_df<PAIR_BS, PAIR_TJ><<<grid, PAIR_BS, 0, s>>>(rec, n, shape.j_per_split, eps2, part);
}

int potential_blocks_per_sm()
{
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_potential_df<PAIR_BS, PAIR_TJ>, PAIR_BS, 0) !=
                cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
    }
    return occ;
}

void launch_aos_to_soa(cudaStream_t s, const double *aos, int n, double *soa, int *err)
{
    if (n <= 0) return;
    k_aos_to_soa<<<cdiv(n, 256), 256, 0, s>>>(aos, n, soa, err);
}

void launch_soa_to_aos(cudaStream_t s, const double *soa, int n, double *aos)
{
    if (n <= 0) return;
    k_soa_to_aos<<<cdiv(n, 256), 256, 0, s>>>(soa, n, aos);
}

void launch_check_mass(cudaStream_t s, const double *m, int n, int *err)
{
    if (n <= 0) return;
    k_check_mass<<<cdiv(n, 256), 256, 0, s>>>(m, n, err);
}

void launch_cluster_energy(cudaStream_t s, const int64_t *offsets, int n_clusters, const double *x,
                           const double *v, const double *m, int N, double eps2, double *out)
{
    if (n_clusters <= 0) return;
    k_cluster_energy<<<n_clusters, 256, 0, s>>>(offsets, x, v, m, N, eps2, out);
}

void launch_energy_reduce(cudaStream_t s, const double *x, const double *v, const double *m, int N,
                          const double *part, int nsplit, double *out)
{
    k_energy_reduce<<<1, 1024, 0, s>>>(x, v, m, N, part, nsplit, out);
}

}  // namespace frost
