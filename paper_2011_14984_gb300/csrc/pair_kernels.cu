// Grid kernels of the HHS-FSI pair passes for sm_103a.
//
//   acc   : a_i = G sum_j m_j x_ji / r_ji^3                       (Eq. acc-newton)
//   grad  : g_i = 2G sum_j m_j r^-5 (r^2 a_ji - 3 (x_ji . a_ji) x_ji) (Eq. acc-gradient-g)
//   tstep : tau_i = eta min_j min(t_ff s(d_ff), t_fb s(d_fb))       (Sec. 4, Eq. time-step-factor)
//
// Work decomposition: a 2-D grid, blockIdx.x over blocks of active particles (i), blockIdx.y
// over contiguous chunks of the source list (j-split).  Each block runs one per-i-block body
// of pair_bodies.cuh over its j-chunk; the partial results per split go to
// part[split][comp][i] and are combined in a fixed order by the finalize kernels, so results
// are deterministic.
//
// Mixed precision: separations are formed from float-float positions, the pair body runs in
// FP32, and the per-tile FP32 partial sums are folded into a TwoSum-compensated (hi, lo)
// FP32 accumulator, converted to FP64 once per block.  The gradient needs accurate
// accelerations (a_j - a_i amplifies their rounding noise): the Newtonian pass that precedes
// it takes a Newton-refined rsqrt and sums each particle's few dominant terms (above 1/16 of
// max_j m_j / r^3, from a prepass) in double-float, and so does the gradient.
//
// The i = j term is excluded by list position: only tiles that overlap the block's own
// i-range (same-list passes) run the masked loop.  Two distinct particles at zero
// separation produce a non-finite partial that the finalize kernels report.
#include "pair_bodies.cuh"

namespace frost {
namespace {

using namespace dev;

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------------------------
// pack kernels
// ------------------------------------------------------------------------------------
__global__ void k_pack_pos_mixed(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                 const double *__restrict__ m, int N, float4 *__restrict__ rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_pos_mixed_one(k, list, n, x, m, N, rec);
}

__global__ void k_pack_grad_mixed(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                  const double *__restrict__ m, int N, const double *__restrict__ acc,
                                  float4 *__restrict__ rec, const uint32_t *__restrict__ hot)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_grad_mixed_one(k, list, n, x, m, N, acc, rec, hot);
}

__global__ void k_pack_tstep_mixed(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                   const double *__restrict__ v, const double *__restrict__ m, int N,
                                   double G, float4 *__restrict__ rec, const double *__restrict__ acc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_tstep_mixed_one(k, list, n, x, v, m, N, G, rec, acc);
}

__global__ void k_pack_pos_fp64(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                const double *__restrict__ m, int N, double4_32a *__restrict__ rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_pos_fp64_one(k, list, n, x, m, N, rec);
}

__global__ void k_pack_grad_fp64(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                 const double *__restrict__ m, int N, const double *__restrict__ acc,
                                 double4_32a *__restrict__ rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_grad_fp64_one(k, list, n, x, m, N, acc, rec);
}

__global__ void k_pack_tstep_fp64(const int32_t *__restrict__ list, int n, const double *__restrict__ x,
                                  const double *__restrict__ v, const double *__restrict__ m, int N,
                                  double G, double4_32a *__restrict__ rec, const double *__restrict__ acc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pack_tstep_fp64_one(k, list, n, x, v, m, N, G, rec, acc);
}

// ------------------------------------------------------------------------------------
// grid pair kernels: one (i-block, j-split) per block
// ------------------------------------------------------------------------------------
template <int BS, int ILP, int TJ, bool WMAX, bool NEWTON = false, bool DEFER = false>
__global__ void __launch_bounds__(BS) k_acc_mixed(const float4 *__restrict__ irec,
                                                  const float4 *__restrict__ jrec, int n_a,
                                                  int n_s, int j_per_split, int self_pass,
                                                  float eps2, double *__restrict__ part,
                                                  float *__restrict__ wpart,
                                                  const float *__restrict__ wmax = nullptr, double eps2d = 0.0,
                                                  const int32_t *__restrict__ jlist = nullptr,
                                                  const double *__restrict__ mstore = nullptr)
{
    const int ibase = blockIdx.x * (BS * ILP);
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    double res[ILP][3];
    float wres[ILP];
    acc_mixed_body<BS, ILP, TJ, WMAX, NEWTON, DEFER>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eps2, res, wres,
                                                     wmax, eps2d, jlist, mstore);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + threadIdx.x;
        if (i < n_a) {
            double *p = part + (size_t)blockIdx.y * 3 * n_a;
            p[i] = res[k][0];
            p[n_a + i] = res[k][1];
            p[2 * n_a + i] = res[k][2];
            if (WMAX) wpart[(size_t)blockIdx.y * n_a + i] = wres[k];
        }
    }
}

// wmax[i] = max over the splits of max_j m_j / r^3 (wmax zeroed before; non-negative floats
// order as their bit patterns, so the maximum is an integer atomicMax)
template <int BS, int ILP, int TJ>
__global__ void __launch_bounds__(BS) k_wmax_mixed(const float4 *__restrict__ irec,
                                                   const float4 *__restrict__ jrec, int n_a, int n_s,
                                                   int j_per_split, int self_pass, float eps2,
                                                   float *__restrict__ wmax)
{
    const int ibase = blockIdx.x * (BS * ILP);
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    float wres[ILP];
    wmax_mixed_body<BS, ILP, TJ>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eps2, wres);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + threadIdx.x;
        if (i < n_a) atomicMax((int *)&wmax[i], __float_as_int(wres[k]));
    }
}

template <int BS, int ILP, int TJ>
__global__ void __launch_bounds__(BS, 512 / BS) k_grad_mixed(const float4 *__restrict__ irec,
                                                   const float4 *__restrict__ jrec, int n_a,
                                                   int n_s, int j_per_split, int self_pass,
                                                   double eps2d, const float *__restrict__ wmax,
                                                   double *__restrict__ part)
{
    const int ibase = blockIdx.x * (BS * ILP);
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    double res[ILP][3];
    grad_mixed_body<BS, ILP, TJ, true>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eps2d, wmax, res);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + threadIdx.x;
        if (i < n_a) {
            double *p = part + (size_t)blockIdx.y * 3 * n_a;
            p[i] = res[k][0];
            p[n_a + i] = res[k][1];
            p[2 * n_a + i] = res[k][2];
        }
    }
}

template <int BS, int ILP, int TJ, int SYM>
__global__ void __launch_bounds__(BS) k_tstep_mixed(const float4 *__restrict__ irec,
                                                    const float4 *__restrict__ jrec, int n_a,
                                                    int n_s, int j_per_split, int self_pass,
                                                    float eta, double *__restrict__ part,
                                                    int *__restrict__ err)
{
    const int ibase = blockIdx.x * (BS * ILP);
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    float best[ILP], minr2[ILP];
    tstep_mixed_body<BS, ILP, TJ, SYM>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eta, best, minr2);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + threadIdx.x;
        if (i < n_a) {
            part[(size_t)blockIdx.y * n_a + i] = (double)best[k];
            if (minr2[k] == 0.f) atomicOr(err, ERR_COINCIDENT);
        }
    }
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_acc_fp64(const double4_32a *__restrict__ irec,
                                                 const double4_32a *__restrict__ jrec, int n_a,
                                                 int n_s, int j_per_split, int self_pass,
                                                 double eps2, double *__restrict__ part)
{
    const int ibase = blockIdx.x * BS;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    double res[3];
    acc_fp64_body<BS, TJ>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eps2, res);
    const int i = ibase + threadIdx.x;
    if (i < n_a) {
        double *p = part + (size_t)blockIdx.y * 3 * n_a;
        p[i] = res[0];
        p[n_a + i] = res[1];
        p[2 * n_a + i] = res[2];
    }
}

template <int BS, int TJ>
__global__ void __launch_bounds__(BS) k_grad_fp64(const double4_32a *__restrict__ irec,
                                                  const double4_32a *__restrict__ jrec, int n_a,
                                                  int n_s, int j_per_split, int self_pass,
                                                  double eps2, double *__restrict__ part)
{
    const int ibase = blockIdx.x * BS;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    double res[3];
    grad_fp64_body<BS, TJ>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eps2, res);
    const int i = ibase + threadIdx.x;
    if (i < n_a) {
        double *p = part + (size_t)blockIdx.y * 3 * n_a;
        p[i] = res[0];
        p[n_a + i] = res[1];
        p[2 * n_a + i] = res[2];
    }
}

template <int BS, int TJ, int SYM>
__global__ void __launch_bounds__(BS) k_tstep_fp64(const double4_32a *__restrict__ irec,
                                                   const double4_32a *__restrict__ jrec, int n_a,
                                                   int n_s, int j_per_split, int self_pass,
                                                   double eta, double *__restrict__ part,
                                                   int *__restrict__ err)
{
    const int ibase = blockIdx.x * BS;
    const int jb = blockIdx.y * j_per_split;
    const int je = min(n_s, jb + j_per_split);
    double best, minr2;
    tstep_fp64_body<BS, TJ, SYM>(irec, jrec, n_a, n_s, ibase, jb, je, self_pass, eta, best, minr2);
    const int i = ibase + threadIdx.x;
    if (i < n_a) {
        part[(size_t)blockIdx.y * n_a + i] = best;
        if (minr2 == 0.0) atomicOr(err, ERR_COINCIDENT);
    }
}

// ------------------------------------------------------------------------------------
// finalisation
// ------------------------------------------------------------------------------------
// sum over the splits of part[p][c][i] (stride = 3 n): four interleaved partial sums, so that
// the loads of a long split list overlap; the association is fixed (deterministic)
__device__ __forceinline__ double split_sum(const double *__restrict__ q, int nsplit, size_t stride)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int p = 0;
    for (; p + 4 <= nsplit; p += 4) {
        s0 += q[(size_t)p * stride];
        s1 += q[(size_t)(p + 1) * stride];
        s2 += q[(size_t)(p + 2) * stride];
        s3 += q[(size_t)(p + 3) * stride];
    }
    for (; p < nsplit; ++p) s0 += q[(size_t)p * stride];
    return (s0 + s1) + (s2 + s3);
}

__global__ void k_finalize_vec(const double *__restrict__ part, int nsplit, int n, double scale,
                               double *__restrict__ out_soa, double *__restrict__ out_aos,
                               int *__restrict__ err, int badbit, KickArgs kick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    const int gi = (kick.v || kick.store) ? (kick.list ? kick.list[i] : i) : 0;
    for (int c = 0; c < 3; ++c) {
        double s = split_sum(part + (size_t)c * n + i, nsplit, (size_t)3 * n);
        s *= scale;
        ok = ok && isfinite(s);
        if (out_soa) out_soa[(size_t)c * n + i] = s;
        if (out_aos) out_aos[(size_t)i * 3 + c] = s;
        // the kick that follows the pass: the roundings of k_kick (no contraction)
        if (kick.v) kick.v[(size_t)c * kick.N + gi] = __dadd_rn(kick.v[(size_t)c * kick.N + gi], __dmul_rn(kick.dt, s));
        if (kick.store) kick.store[(size_t)c * kick.N + gi] = s;
    }
    if (!ok) atomicOr(err, badbit);
}

__global__ void k_finalize_grad(const double *__restrict__ part, int nsplit, int n, double scale,
                                const double *__restrict__ a_soa, double c,
                                double *__restrict__ at_soa, double *__restrict__ at_aos,
                                double *__restrict__ g_aos, int *__restrict__ err, int badbit,
                                const double *__restrict__ part2, int nsplit2, KickArgs kick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    const int gi = kick.v ? (kick.list ? kick.list[i] : i) : 0;
    for (int k = 0; k < 3; ++k) {
        double s = split_sum(part + (size_t)k * n + i, nsplit, (size_t)3 * n);
        for (int p = 0; p < nsplit2; ++p) s += part2[((size_t)p * 3 + k) * n + i];
        const double g = scale * s;
        const double at = a_soa[(size_t)k * n + i] + c * g;
        ok = ok && isfinite(at) && isfinite(g);
        if (at_soa) at_soa[(size_t)k * n + i] = at;
        if (at_aos) at_aos[(size_t)i * 3 + k] = at;
        if (g_aos) g_aos[(size_t)i * 3 + k] = g;
        if (kick.v) kick.v[(size_t)k * kick.N + gi] = __dadd_rn(kick.v[(size_t)k * kick.N + gi], __dmul_rn(kick.dt, at));
    }
    if (!ok) atomicOr(err, badbit);
}

__global__ void k_finalize_tau(const double *__restrict__ part, int nsplit, int n, double eta,
                               double *__restrict__ tau, int *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double b0 = INFINITY, b1 = INFINITY;
    int p = 0;
    for (; p + 2 <= nsplit; p += 2) {
        b0 = fmin(b0, part[(size_t)p * n + i]);
        b1 = fmin(b1, part[(size_t)(p + 1) * n + i]);
    }
    if (p < nsplit) b0 = fmin(b0, part[(size_t)p * n + i]);
    const double b = fmin(b0, b1);
    const double t = eta * b;
    if (!(t > 0.0)) atomicOr(err, ERR_NONFINITE);  // NaN or non-positive step
    tau[i] = t;
}

// Cached occupancy (blocks per SM) of each pair-kernel instantiation.
template <typename K>
int occupancy_of(K kernel, int bs, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, bs, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
void launch_pack_pos_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                           const double *m, int N, float4 *rec)
{
    if (n <= 0) return;
    k_pack_pos_mixed<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, m, N, rec);
}
void launch_pack_grad_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                            const double *m, int N, const double *acc, float4 *rec, const uint32_t *hot)
{
    if (n <= 0) return;
    k_pack_grad_mixed<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, m, N, acc, rec, hot);
}
void launch_pack_tstep_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                             const double *v, const double *m, int N, double G, float4 *rec, const double *acc)
{
    if (n <= 0) return;
    k_pack_tstep_mixed<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, v, m, N, G, rec, acc);
}
void launch_pack_pos_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                          const double *m, int N, double4_32a *rec)
{
    if (n <= 0) return;
    k_pack_pos_fp64<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, m, N, rec);
}
void launch_pack_grad_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                           const double *m, int N, const double *acc, double4_32a *rec)
{
    if (n <= 0) return;
    k_pack_grad_fp64<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, m, N, acc, rec);
}
void launch_pack_tstep_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                            const double *v, const double *m, int N, double G, double4_32a *rec,
                            const double *acc)
{
    if (n <= 0) return;
    k_pack_tstep_fp64<<<cdiv(n, 256), 256, 0, s>>>(list, n, x, v, m, N, G, rec, acc);
}

int pair_i_per_block(bool mixed) { return mixed ? PAIR_BS * PAIR_ILP : PAIR_BS; }

int pair_blocks_per_sm(int kind, bool mixed, bool small)
{
    static int cache[3][2] = {{0, 0}, {0, 0}, {0, 0}}, cache_small[3] = {0, 0, 0};
    if (small) {
        constexpr int B = PAIR_BS_SMALL, L = PAIR_ILP, T = PAIR_TJ_SMALL;
        int &c = cache_small[kind];
        if (c) return c;
        if (kind == PASS_ACC)
            c = std::min(occupancy_of(k_acc_mixed<B, L, T, false>, B, 0),
                         occupancy_of(k_acc_mixed<B, L, T, false, true, true>, B, 0));
        else if (kind == PASS_GRAD)
            c = occupancy_of(k_grad_mixed<B, L, T>, B, 0);
        else
            c = occupancy_of(k_tstep_mixed<B, L, T, 0>, B, 0);
        return c;
    }
    int &c = cache[kind][mixed ? 1 : 0];
    if (c) return c;
    if (kind == PASS_ACC)
        c = mixed ? std::min(occupancy_of(k_acc_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, false>, PAIR_BS, 0),
                             occupancy_of(k_acc_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, false, true, true>, PAIR_BS, 0))
                  : occupancy_of(k_acc_fp64<PAIR_BS, PAIR_TJ>, PAIR_BS, 0);
    else if (kind == PASS_GRAD)
        c = mixed ? occupancy_of(k_grad_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ>, PAIR_BS, 0)
                  : occupancy_of(k_grad_fp64<PAIR_BS, PAIR_TJ>, PAIR_BS, 0);
    else
        c = mixed ? occupancy_of(k_tstep_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, 0>, PAIR_BS, 0)
                  : occupancy_of(k_tstep_fp64<PAIR_BS, PAIR_TJ, 0>, PAIR_BS, 0);
    return c;
}

SplitShape choose_shape(int n_a, int n_s, int i_per_block, int blocks_per_sm, int n_sm, int max_waves, int tj)
{
    SplitShape sh;
    sh.nblk_i = (n_a + i_per_block - 1) / i_per_block;
    if (sh.nblk_i < 1) sh.nblk_i = 1;
    const long long cap = (long long)blocks_per_sm * n_sm;
    const int tiles = (n_s + tj - 1) / tj;
    int best_split = 1;
    double best_eff = -1.0;
    // at most max_waves full waves of blocks in total, each split at least one tile
    const int max_split =
        (int)std::max<long long>(1, std::min<long long>(tiles, ((long long)max_waves * cap) / sh.nblk_i));
    for (int ns = 1; ns <= max_split; ++ns) {
        const int tps = (tiles + ns - 1) / ns;                 // tiles per split
        const int nsp = (tiles + tps - 1) / tps;                // splits actually used
        const long long total = (long long)sh.nblk_i * nsp;
        const long long waves = (total + cap - 1) / cap;
        // slot use of the waves, discounted by a per-block overhead of ~1/2 tile
        const double eff = (double)total * tps / ((double)waves * cap * (tps + 0.5));
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_split = ns;
        }
    }
    const int tps = (tiles + best_split - 1) / best_split;
    sh.j_per_split = std::max(1, tps) * tj;
    sh.nsplit = std::max(1, (n_s + sh.j_per_split - 1) / sh.j_per_split);
    return sh;
}

void launch_acc(cudaStream_t s, bool mixed, const PairArgs &a)
{
    const dim3 grid(a.shape.nblk_i, a.shape.nsplit);
    if (mixed && a.shape.small) {
        constexpr int B = PAIR_BS_SMALL, L = PAIR_ILP, T = PAIR_TJ_SMALL;
        if (a.accurate)
            k_acc_mixed<B, L, T, false, true, true><<<grid, B, 0, s>>>(
                (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split, a.self_pass,
                (float)a.eps2, a.part, nullptr, a.wmax, a.eps2, a.jlist, a.m);
        else
            k_acc_mixed<B, L, T, false><<<grid, B, 0, s>>>((const float4 *)a.irec, (const float4 *)a.jrec, a.n_a,
                                                           a.n_s, a.shape.j_per_split, a.self_pass, (float)a.eps2,
                                                           a.part, nullptr);
    } else if (mixed && a.accurate) {
        k_acc_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, false, true, true><<<grid, PAIR_BS, 0, s>>>(
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, (float)a.eps2, a.part, nullptr, a.wmax, a.eps2, a.jlist, a.m);
    } else if (mixed) {
        k_acc_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, false><<<grid, PAIR_BS, 0, s>>>(
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, (float)a.eps2, a.part, nullptr);
    } else {
        k_acc_fp64<PAIR_BS, PAIR_TJ><<<grid, PAIR_BS, 0, s>>>(
            (const double4_32a *)a.irec, (const double4_32a *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, a.eps2, a.part);
    }
}

void launch_wmax(cudaStream_t s, const PairArgs &a, float *wmax)
{
    cudaMemsetAsync(wmax, 0, sizeof(float) * a.n_a, s);
    const dim3 grid(a.shape.nblk_i, a.shape.nsplit);
    if (a.shape.small) {
        k_wmax_mixed<PAIR_BS_SMALL, PAIR_ILP, PAIR_TJ_SMALL><<<grid, PAIR_BS_SMALL, 0, s>>>(
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split, a.self_pass,
            (float)a.eps2, wmax);
        return;
    }
    k_wmax_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ><<<grid, PAIR_BS, 0, s>>>(
        (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split, a.self_pass,
        (float)a.eps2, wmax);
}

void launch_grad(cudaStream_t s, bool mixed, const PairArgs &a)
{
    const dim3 grid(a.shape.nblk_i, a.shape.nsplit);
    if (mixed && a.shape.small)
        k_grad_mixed<PAIR_BS_SMALL, PAIR_ILP, PAIR_TJ_SMALL><<<grid, PAIR_BS_SMALL, 0, s>>>(
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, a.eps2, a.wmax, a.part);
    else if (mixed)
        k_grad_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ><<<grid, PAIR_BS, 0, s>>>(
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, a.eps2, a.wmax, a.part);
    else
        k_grad_fp64<PAIR_BS, PAIR_TJ><<<grid, PAIR_BS, 0, s>>>(
            (const double4_32a *)a.irec, (const double4_32a *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,
            a.self_pass, a.eps2, a.part);
}

void launch_tstep(cudaStream_t s, bool mixed, const PairArgs &a, double eta, int sym, int *err)
{
    const dim3 grid(a.shape.nblk_i, a.shape.nsplit);
#define FROST_TSTEP_CASE(SYMV)                                                                    \
    if (mixed && a.shape.small)                                                                   \
        k_tstep_mixed<PAIR_BS_SMALL, PAIR_ILP, PAIR_TJ_SMALL, SYMV><<<grid, PAIR_BS_SMALL, 0, s>>>( \
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,    \
            a.self_pass, (float)eta, a.part, err);                                                \
    else if (mixed)                                                                               \
        k_tstep_mixed<PAIR_BS, PAIR_ILP, PAIR_TJ, SYMV><<<grid, PAIR_BS, 0, s>>>(                 \
            (const float4 *)a.irec, (const float4 *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,    \
            a.self_pass, (float)eta, a.part, err);                                                \
    else                                                                                          \
        k_tstep_fp64<PAIR_BS, PAIR_TJ, SYMV><<<grid, PAIR_BS, 0, s>>>(                            \
            (const double4_32a *)a.irec, (const double4_32a *)a.jrec, a.n_a, a.n_s, a.shape.j_per_split,  \
            a.self_pass, eta, a.part, err);
    // sym & 3: symmetrisation factor; sym & 4: exact fly-by derivative (records with a)
    switch (sym) {
    case 0: FROST_TSTEP_CASE(0) break;
    case 1: FROST_TSTEP_CASE(1) break;
    case 4: FROST_TSTEP_CASE(4) break;
    case 5: FROST_TSTEP_CASE(5) break;
    case 6: FROST_TSTEP_CASE(6) break;
    default: FROST_TSTEP_CASE(2) break;
    }
#undef FROST_TSTEP_CASE
}

void launch_finalize_vec(cudaStream_t s, const double *part, int nsplit, int n, double scale,
                         double *out_soa, double *out_aos, int *err, int badbit, KickArgs kick)
{
    if (n <= 0) return;
    k_finalize_vec<<<cdiv(n, 256), 256, 0, s>>>(part, nsplit, n, scale, out_soa, out_aos, err, badbit, kick);
}

void launch_finalize_grad(cudaStream_t s, const double *part, int nsplit, int n, double scale,
                          const double *a_soa, double c, double *at_soa, double *at_aos,
                          double *g_aos, int *err, int badbit, const double *part2, int nsplit2,
                          KickArgs kick)
{
    if (n <= 0) return;
    k_finalize_grad<<<cdiv(n, 256), 256, 0, s>>>(part, nsplit, n, scale, a_soa, c, at_soa, at_aos,
                                                  g_aos, err, badbit, part2, part2 ? nsplit2 : 0, kick);
}

void launch_finalize_tau(cudaStream_t s, const double *part, int nsplit, int n, double eta,
                         double *tau, int *err)
{
    if (n <= 0) return;
    k_finalize_tau<<<cdiv(n, 256), 256, 0, s>>>(part, nsplit, n, eta, tau, err);
}

}  // namespace frost
