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
//   * k_acc_refine recomputes their accelerations with the dominant terms (m_k / r^3 above a
//     quarter of the largest) in FP64 from the FP64 store, so that the partners' mutual forces
//     are as consistent as in FP64, and marks them in a bit mask;
//   * the gradient pass zeroes their masses in its FP32 records and k_grad_hot sums their
//     terms in FP64 for every active particle, into separate split partials.
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

// deterministic block sum of three doubles; the result is valid in thread 0
__device__ void block_sum3(double (&v)[3])
{
    __shared__ double s_r[HOT_BS / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    __syncthreads();
    if (lane == 0)
        for (int c = 0; c < 3; ++c) s_r[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int w = 0; w < HOT_BS / 32; ++w) s += s_r[w][c];
            v[c] = s;
        }
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
__device__ __forceinline__ int nth_hot(const unsigned *words, int q)
{
    for (int w = 0; w < HOT_BS / 32; ++w) {
        const unsigned bits = words[w];
        const int c = __popc(bits);
        if (q < c) {
            unsigned b = bits;
            for (int k = 0; k < q; ++k) b &= b - 1u;
            return w * 32 + __ffs(b) - 1;
        }
        q -= c;
    }
    return 0;
}

// one thread's share of the refined acceleration of target t: the sources j0, j0 + dj, ...;
// FP32 pair terms on the three-way split records, except up to GRAD_SLOTS terms with
// m_j / r^3 > thr, which are evaluated in FP64 from the particle store
__device__ void refine_partial(int t, int j0, int dj, const float4 *__restrict__ irec,
                               const float4 *__restrict__ jrec, int n_a, int n_s, int self_pass,
                               const int32_t *__restrict__ Alist, const int32_t *__restrict__ Blist,
                               const double *__restrict__ x, const double *__restrict__ m, int N,
                               double eps2d, float thr, double (&r)[3])
{
    const float eps2 = (float)eps2d;
    const float4 q0 = irec[t], q1 = irec[n_a + t], q2 = irec[2 * n_a + t];
    int nb = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    float H[3] = {0.f, 0.f, 0.f}, L[3] = {0.f, 0.f, 0.f}, s[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    for (int j = j0; j < n_s; j += dj) {
        if (self_pass && j == t) continue;
        const float4 J0 = jrec[j], J1 = jrec[n_s + j], J2 = jrec[2 * n_s + j];
        const float dx = ((J0.x - q0.x) + (J1.x - q1.x)) + (J2.x - q2.x);
        const float dy = ((J0.y - q0.y) + (J1.y - q1.y)) + (J2.y - q2.y);
        const float dz = ((J0.z - q0.z) + (J1.z - q1.z)) + (J2.z - q2.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        float y = rsqrtf(r2);
        const float hy = (0.5f * r2) * y;
        y = fmaf(y, fmaf(-hy, y, 0.5f), y);
        const float wt = J0.w * y * (y * y);
        if (wt > thr && nb < GRAD_SLOTS) {
            if (nb == 0) b0 = j;
            else if (nb == 1) b1 = j;
            else if (nb == 2) b2 = j;
            else b3 = j;
            ++nb;
            continue;
        }
        s[0] = fmaf(wt, dx, s[0]);
        s[1] = fmaf(wt, dy, s[1]);
        s[2] = fmaf(wt, dz, s[2]);
        if (++cnt == 16) {
            for (int c = 0; c < 3; ++c) {
                fold2(H[c], L[c], s[c]);
                s[c] = 0.f;
            }
            cnt = 0;
        }
    }
    for (int c = 0; c < 3; ++c) {
        fold2(H[c], L[c], s[c]);
        r[c] = (double)H[c] + (double)L[c];
    }
    const int gi = Alist ? Alist[t] : t;
    const double xi = x[gi], yi = x[N + gi], zi = x[2 * N + gi];
    for (int q = 0; q < nb; ++q) {
        const int j = (q == 0) ? b0 : (q == 1) ? b1 : (q == 2) ? b2 : b3;
        const int gj = Blist ? Blist[j] : j;
        const double ddx = x[gj] - xi, ddy = x[N + gj] - yi, ddz = x[2 * N + gj] - zi;
        const double rr2 = fma(ddx, ddx, fma(ddy, ddy, fma(ddz, ddz, eps2d)));
        const double ri = rsqrt(rr2);
        const double ww = m[gj] * (ri * ri * ri);
        r[0] = fma(ww, ddx, r[0]);
        r[1] = fma(ww, ddy, r[1]);
        r[2] = fma(ww, ddz, r[2]);
    }
}

// Marks the hot particles of a finished accurate Newtonian pass of A against B (mask bit k of
// word k / 32) and recomputes their accelerations: FP32 pair terms on the three-way split
// records of that pass, except up to GRAD_SLOTS terms per thread with m_j / r^3 above
// wmax_k / 4, which are evaluated in FP64 from the particle store.  The threshold is
// HOT_KAPPA x the larger median edge of hist (n_a values of this pass) and hist2 (n2 values
// of the companion pass of B against A, or NULL).  One block per 256 particles: with at most
// two hot particles the whole block refines each, otherwise one warp per hot particle; the
// sums run in a fixed order either way.
__global__ void __launch_bounds__(HOT_BS) k_acc_refine(
    const float4 *__restrict__ irec, const float4 *__restrict__ jrec, int n_a, int n_s, int self_pass,
    const int32_t *__restrict__ Alist, const int32_t *__restrict__ Blist, const double *__restrict__ x,
    const double *__restrict__ m, int N, double G, double eps2d, const float *__restrict__ wmax,
    const unsigned *__restrict__ hist, const unsigned *__restrict__ hist2, int n2,
    double *__restrict__ out_soa, double *__restrict__ out_aos, uint32_t *__restrict__ mask)
{
    __shared__ float s_thr;
    __shared__ unsigned s_words[HOT_BS / 32];
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
    if (k < n_a) hot = acc_norm(out_soa[k], out_soa[n_a + k], out_soa[2 * n_a + k]) > s_thr;
    const unsigned word = __ballot_sync(0xffffffffu, hot);
    if (lane == 0) {
        s_words[warp] = word;
        if (base + warp * 32 < n_a) mask[(base >> 5) + warp] = word;
    }
    __syncthreads();
    int nhot = 0;
    for (int w = 0; w < HOT_BS / 32; ++w) nhot += __popc(s_words[w]);
    if (nhot <= 2) {
        // few targets: each one by the whole block
        for (int q = 0; q < nhot; ++q) {
            const int t = base + nth_hot(s_words, q);
            double r[3];
            refine_partial(t, tid, HOT_BS, irec, jrec, n_a, n_s, self_pass, Alist, Blist, x, m, N, eps2d,
                           0.25f * wmax[t], r);
            block_sum3(r);
            if (tid == 0)
                for (int c = 0; c < 3; ++c) {
                    const double a = G * r[c];
                    out_soa[(size_t)c * n_a + t] = a;
                    if (out_aos) out_aos[(size_t)t * 3 + c] = a;
                }
            __syncthreads();
        }
    } else {
        // many targets: one warp each, no block barrier
        for (int q = warp; q < nhot; q += HOT_BS / 32) {
            const int t = base + nth_hot(s_words, q);
            double r[3];
            refine_partial(t, lane, 32, irec, jrec, n_a, n_s, self_pass, Alist, Blist, x, m, N, eps2d,
                           0.25f * wmax[t], r);
            for (int c = 0; c < 3; ++c)
                for (int o = 16; o > 0; o >>= 1) r[c] += __shfl_xor_sync(0xffffffffu, r[c], o);
            if (lane == 0)
                for (int c = 0; c < 3; ++c) {
                    const double a = G * r[c];
                    out_soa[(size_t)c * n_a + t] = a;
                    if (out_aos) out_aos[(size_t)t * 3 + c] = a;
                }
        }
    }
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
                    for (int c = 0; c < 3; ++c) g[c] = df::add(g[c], df::mul(w, df::sub(A[c], df::mul(t3, d[c]))));
                }
            }
            __syncthreads();
        }
    }
    if (i < n_a)
        for (int c = 0; c < 3; ++c) part[((size_t)sp * 3 + c) * n_a + i] = df::to_double(g[c]);
}

void launch_acc_hist(cudaStream_t s, const double *a_soa, int n, unsigned *hist)
{
    if (n <= 0) return;
    const int blocks = std::min((n + HOT_BS - 1) / HOT_BS, 1024);
    k_acc_hist<<<blocks, HOT_BS, 0, s>>>(a_soa, n, hist);
}

void launch_acc_refine(cudaStream_t s, const float4 *irec, const float4 *jrec, int n_a, int n_s,
                       int self_pass, const int32_t *A, const int32_t *B, const double *x,
                       const double *m, int N, double G, double eps2, const float *wmax,
                       const unsigned *hist, const unsigned *hist2, int n2, double *out_soa,
                       double *out_aos, uint32_t *mask)
{
    if (n_a <= 0) return;
    k_acc_refine<<<(n_a + HOT_BS - 1) / HOT_BS, HOT_BS, 0, s>>>(irec, jrec, n_a, n_s, self_pass, A, B, x,
                                                                m, N, G, eps2, wmax, hist, hist2, n2,
                                                                out_soa, out_aos, mask);
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
