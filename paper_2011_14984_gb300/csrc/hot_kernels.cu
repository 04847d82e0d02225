// Hot sources of the mixed-precision gradient pass.
//
// The gradient of particle i sums m_j K(x_ji) (a_j - a_i) with K(x) = r^-3 - 3 r^-5 x x^T
// (Eq. acc-gradient-g).  A source whose acceleration is far above the typical one -- a member
// of a hard binary -- gives a large term, and the terms of the two partners cancel to a
// remainder smaller by (separation within the pair) / (distance to i).  A relative rounding
// error of 1e-7 in such a term, or in such an a_j, is amplified by the inverse of that ratio,
// so FP32 pair arithmetic cannot hold the gradient of the other particles to 1e-6.
//
// The size of a_ji in a pass is set by the typical |a| of both lists, so sources with
// |a_j| > HOT_KAPPA x (upper edge of the histogram bin holding the median |a| of the active
// list, or of the source list if that is larger) are "hot":
//   * k_hot_mask marks them in a bit mask (their accelerations are already accurate: the
//     Newtonian pass that feeds a gradient sums its dominant terms in double-float with the
//     FP64 masses, so the partners' mutual forces are as consistent as in FP64);
//   * the gradient pass zeroes their masses in its FP32 records and k_grad_hot sums their
//     terms in double-float for every active particle, into separate split partials.
// The classification depends only on the accelerations, so the results stay deterministic;
// with no hot source both kernels only read the mask and write zeros.
#include "df_arith.cuh"
#include "frost_internal.cuh"
#include "pair_bodies.cuh"

namespace frost {

using namespace dev;

namespace {

constexpr int HOT_BS = 256;
constexpr int HOT_WORDS = 128;  // mask words gathered per chunk by k_grad_hot

// bin of |f|: exponent and the two leading mantissa bits (4 bins per octave); the sign bit of
// a NaN is dropped, so the bin is always below HOT_BINS
__device__ __forceinline__ unsigned hot_bin(float f) { return (__float_as_uint(f) & 0x7fffffffu) >> 21; }

// |a| as the classification sees it (FP32 of the FP64 norm)
__device__ __forceinline__ float acc_norm(double ax, double ay, double az)
{
    return (float)sqrt(fma(ax, ax, fma(ay, ay, az * az)));
}

// the upper edge of the bin holding the median of the n counted values; called by a whole
// warp, the result is returned to every lane
__device__ float median_edge(const unsigned *__restrict__ hist, int n)
{
    const int lane = threadIdx.x & 31;
    unsigned s = 0;
    // lane sums its 32 bins in a rotated order, so that a histogram in shared memory is read
    // without bank conflicts
    for (int q = 0; q < 32; ++q) s += hist[lane * 32 + ((q + lane) & 31)];
    unsigned incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned r = (unsigned)(n + 1) / 2;  // 1-based rank of the median
    const unsigned ball = __ballot_sync(0xffffffffu, incl >= r);
    if (ball == 0u) return INFINITY;
    const int L = __ffs(ball) - 1;
    float thr = INFINITY;
    if (lane == L) {
        unsigned c = incl - s;
        int b = lane * 32 + 31;
        for (int q = 0; q < 32; ++q) {
            c += hist[lane * 32 + q];
            if (c >= r) {
                b = lane * 32 + q;
                break;
            }
        }
        // bins from 1019 up reach the top octave, infinities and NaNs: nothing is hot
        thr = (b >= 1019) ? INFINITY : __uint_as_float((unsigned)(b + 1) << 21);
    }
    return __shfl_sync(0xffffffffu, thr, L);
}

// exclusive block scan of one value per thread (HOT_BS threads); returns the prefix and the
// block total in *total
__device__ int block_scan(int v, int *total)
{
    __shared__ int s_w[HOT_BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < HOT_BS / 32; ++w) {
        const int c = s_w[w];
        before += (w < warp) ? c : 0;
        all += c;
    }
    *total = all;
    return before + incl - v;
}

}  // namespace

// Histogram of the acceleration norms of a finished Newtonian pass: one count per particle in
// hist[hot_bin(|a_i|)] (HOT_BINS bins, zeroed by the caller).
__global__ void __launch_bounds__(HOT_BS) k_acc_hist(const double *__restrict__ a_soa, int n,
                                                     unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[HOT_BINS];
    for (int b = threadIdx.x; b < HOT_BINS; b += HOT_BS) sh[b] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * HOT_BS + threadIdx.x; i < n; i += gridDim.x * HOT_BS)
        atomicAdd(&sh[hot_bin(acc_norm(a_soa[i], a_soa[n + i], a_soa[2 * n + i]))], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < HOT_BINS; b += HOT_BS)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// position within the block (0..HOT_BS) of the q-th set bit of the block's mask words
// Marks the hot particles of a finished accurate Newtonian pass of A against B: mask bit k
// of word k / 32 is set when |a_k| exceeds HOT_KAPPA x the larger median edge of hist (n_a
// values of this pass) and hist2 (n2 values of the companion pass of B against A, or NULL).
__global__ void __launch_bounds__(HOT_BS) k_hot_mask(const double *__restrict__ a_soa, int n_a,
                                                     const unsigned *__restrict__ hist,
                                                     const unsigned *__restrict__ hist2, int n2,
                                                     uint32_t *__restrict__ mask)
{
    __shared__ float s_thr;
    __shared__ unsigned s_hist[2][HOT_BINS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool two = hist2 && n2 > 0;
    for (int b = tid; b < HOT_BINS; b += HOT_BS) {
        s_hist[0][b] = hist[b];
        if (two) s_hist[1][b] = hist2[b];
    }
    __syncthreads();
    if (warp == 0) {
        float e = median_edge(s_hist[0], n_a);
        if (two) e = fmaxf(e, median_edge(s_hist[1], n2));
        if (lane == 0) s_thr = HOT_KAPPA * e;
    }
    __syncthreads();
    const int base = blockIdx.x * HOT_BS;
    const int k = base + tid;
    bool hot = false;
    if (k < n_a) hot = acc_norm(a_soa[k], a_soa[n_a + k], a_soa[2 * n_a + k]) > s_thr;
    const unsigned word = __ballot_sync(0xffffffffu, hot);
    if (lane == 0 && base + warp * 32 < n_a) mask[(base >> 5) + warp] = word;
}

// Gradient terms of the hot sources of B (mask bits) for every particle of A, in double-float
// arithmetic (df_arith.cuh, about 1e-13 relative per term, well below what the cancellation
// between partners needs; FP64 would run at 1/60 of the FP32 rate):
// part[s][c][i] = sum over the hot j of split s of m_j r^-5 (r^2 a_ji - 3 (x_ji . a_ji) x_ji).
// Positions enter exactly as three FP32 parts, accelerations and masses as double-floats.
// Split s takes the mask words s, s + nsplit, s + 2 nsplit, ... so that hot sources clustered
// in index order still spread over the splits.
__global__ void __launch_bounds__(HOT_BS) k_grad_hot(
    const int32_t *__restrict__ Alist, int n_a, const double *__restrict__ aA,
    const int32_t *__restrict__ Blist, int n_s, const double *__restrict__ aB,
    const uint32_t *__restrict__ mask, int self_pass, const double *__restrict__ x,
    const double *__restrict__ m, int N, double eps2d, int nsplit, double *__restrict__ part)
{
    using df::dfloat;
    __shared__ int s_list[HOT_WORDS * 32];
    // per hot source: x as three parts (9 floats), a as double-floats (6), m (2)
    __shared__ float s_j[17][HOT_BS];
    __shared__ int s_pos[HOT_BS];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * HOT_BS + tid;
    const int sp = blockIdx.y;
    float xi[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    dfloat ai[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (i < n_a) {
        const int gi = Alist ? Alist[i] : i;
        for (int c = 0; c < 3; ++c) {
            df::split3(x[(size_t)c * N + gi], xi[c][0], xi[c][1], xi[c][2]);
            ai[c] = df::from_double(aA[(size_t)c * n_a + i]);
        }
    }
    const dfloat e2 = df::from_double(eps2d);
    dfloat g[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double g64[3] = {0.0, 0.0, 0.0};  // terms outside the FP32 exponent range, in FP64
    const int n_words = (n_s + 31) >> 5;
    const int q_count = (sp < n_words) ? (n_words - sp + nsplit - 1) / nsplit : 0;
    for (int q0 = 0; q0 < q_count; q0 += HOT_WORDS) {
        unsigned bits = 0u;
        int wi = 0;
        if (tid < HOT_WORDS && q0 + tid < q_count) {
            wi = sp + nsplit * (q0 + tid);
            bits = mask[wi];
        }
        int total;
        int o = block_scan(__popc(bits), &total);
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            s_list[o++] = wi * 32 + b;
        }
        __syncthreads();
        for (int t0 = 0; t0 < total; t0 += HOT_BS) {
            const int nt = min(HOT_BS, total - t0);
            if (tid < nt) {
                const int jp = s_list[t0 + tid];
                const int gj = Blist ? Blist[jp] : jp;
                s_pos[tid] = jp;
                for (int c = 0; c < 3; ++c) {
                    df::split3(x[(size_t)c * N + gj], s_j[3 * c][tid], s_j[3 * c + 1][tid], s_j[3 * c + 2][tid]);
                    const dfloat a = df::from_double(aB[(size_t)c * n_s + jp]);
                    s_j[9 + 2 * c][tid] = a.h;
                    s_j[10 + 2 * c][tid] = a.l;
                }
                const dfloat mj = df::from_double(m[gj]);
                s_j[15][tid] = mj.h;
                s_j[16][tid] = mj.l;
            }
            __syncthreads();
            if (i < n_a) {
                for (int u = 0; u < nt; ++u) {
                    if (self_pass && s_pos[u] == i) continue;
                    dfloat d[3], A[3];
                    for (int c = 0; c < 3; ++c) {
                        d[c] = df::sep(s_j[3 * c][u], s_j[3 * c + 1][u], s_j[3 * c + 2][u], xi[c][0], xi[c][1],
                                       xi[c][2]);
                        dfloat aj;
                        aj.h = s_j[9 + 2 * c][u];
                        aj.l = s_j[10 + 2 * c][u];
                        A[c] = df::sub(aj, ai[c]);
                    }
                    const dfloat r2 = df::add(df::add(df::mul(d[0], d[0]), df::mul(d[1], d[1])),
                                              df::add(df::mul(d[2], d[2]), e2));
                    const dfloat ri = df::rsqrt(r2);
                    const dfloat ri2 = df::mul(ri, ri);
                    dfloat mj;
                    mj.h = s_j[15][u];
                    mj.l = s_j[16][u];
                    const dfloat w = df::mul(mj, df::mul(ri2, ri));
                    const dfloat xa = df::add(df::add(df::mul(d[0], A[0]), df::mul(d[1], A[1])), df::mul(d[2], A[2]));
                    const dfloat t3 = df::mul(df::mul_f(xa, 3.f), ri2);
                    dfloat t[3];
                    bool finite = true;
                    for (int c = 0; c < 3; ++c) {
                        t[c] = df::mul(w, df::sub(A[c], df::mul(t3, d[c])));
                        finite = finite && isfinite(t[c].h) && isfinite(t[c].l);
                    }
                    if (finite) {
                        for (int c = 0; c < 3; ++c) g[c] = df::add(g[c], t[c]);
                    } else {
                        // near the pericentre of a hard binary the term exceeds the largest FP32
                        // value: the same term in FP64 from the same parts (they sum exactly)
                        double dd[3], AA[3];
                        for (int c = 0; c < 3; ++c) {
                            dd[c] = ((double)s_j[3 * c][u] + (double)s_j[3 * c + 1][u] + (double)s_j[3 * c + 2][u]) -
                                    ((double)xi[c][0] + (double)xi[c][1] + (double)xi[c][2]);
                            AA[c] = ((double)s_j[9 + 2 * c][u] + (double)s_j[10 + 2 * c][u]) -
                                    ((double)ai[c].h + (double)ai[c].l);
                        }
                        const double rr2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] + eps2d;
                        const double rri = 1.0 / sqrt(rr2);
                        const double ww = ((double)mj.h + (double)mj.l) * rri * rri * rri;
                        const double tt3 = 3.0 * (dd[0] * AA[0] + dd[1] * AA[1] + dd[2] * AA[2]) * rri * rri;
                        for (int c = 0; c < 3; ++c) g64[c] += ww * (AA[c] - tt3 * dd[c]);
                    }
                }
            }
            __syncthreads();
        }
    }
    if (i < n_a)
        for (int c = 0; c < 3; ++c) part[((size_t)sp * 3 + c) * n_a + i] = df::to_double(g[c]) + g64[c];
}

void launch_acc_hist(cudaStream_t s, const double *a_soa, int n, unsigned *hist)
{
    if (n <= 0) return;
    const int blocks = std::min((n + HOT_BS - 1) / HOT_BS, 1024);
    k_acc_hist<<<blocks, HOT_BS, 0, s>>>(a_soa, n, hist);
}

void launch_hot_mask(cudaStream_t s, const double *a_soa, int n_a, const unsigned *hist,
                     const unsigned *hist2, int n2, uint32_t *mask)
{
    if (n_a <= 0) return;
    k_hot_mask<<<(n_a + HOT_BS - 1) / HOT_BS, HOT_BS, 0, s>>>(a_soa, n_a, hist, hist2, n2, mask);
}

int hot_grad_splits(int n_a, int n_s, int n_sm)
{
    const int nblk = (n_a + HOT_BS - 1) / HOT_BS;
    const int n_words = (n_s + 31) / 32;
    int ns = std::max(1, (2 * n_sm) / std::max(1, nblk));
    ns = std::min(ns, HOT_MAX_SPLITS);
    return std::max(1, std::min(ns, n_words));
}

void launch_grad_hot(cudaStream_t s, const int32_t *A, int n_a, const double *aA, const int32_t *B,
                     int n_s, const double *aB, const uint32_t *mask, int self_pass, const double *x,
                     const double *m, int N, double eps2, int nsplit, double *part)
{
    if (n_a <= 0) return;
    const dim3 grid((n_a + HOT_BS - 1) / HOT_BS, nsplit);
    k_grad_hot<<<grid, HOT_BS, 0, s>>>(A, n_a, aA, B, n_s, aB, mask, self_pass, x, m, N, eps2, nsplit,
                                       part);
}

}  // namespace frost
