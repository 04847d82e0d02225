// Single-CTA HHS-FSI subtree solver for sm_103a.
//
// Runs Algorithm hhs-fsi on a set P entirely inside one thread block: time-step pass, stable
// partition, inter-level kicks (kick_sf), FSI steps of the slow set and the recursion into
// the fast set, with an explicit stack in shared memory instead of host round trips.  By
// the HOLD property of the splitting (Sec. 3.1), the subtree of a set only involves the
// particles of that set, so one block can finish it without touching any other particle.
// The host hands every hhs_fsi call whose set is at most a threshold size to this kernel
// (the deep, small levels of the hierarchy, where one kernel launch per pass and a host
// synchronisation per level would dominate).  With an offsets array the same kernel
// advances many independent clusters, one cluster per block.
//
// The pair passes are the same per-i-block bodies as the grid kernels (pair_bodies.cuh),
// here looped over the i-blocks of the set against the whole source list; results are
// therefore the same to rounding (the grid path splits the sources differently).  Every
// block-level helper ends with __syncthreads(); all control decisions are block-uniform.
#include "pair_bodies.cuh"

namespace frost {
namespace {

using namespace dev;

constexpr int SB = 256;           // threads per subtree block
constexpr int SILP = 2;           // i-particles per thread (mixed)
constexpr int STJ = 128;          // source records per shared-memory tile
constexpr int SIB = SB * SILP;    // i-block of the mixed bodies
constexpr int MAXD = SUBTREE_MAX_FRAMES;

struct SubParams {
    double *x, *v;
    const double *m;
    int N;
    double G, eta, eps2;
    int max_depth;
    int *err;
    unsigned long long *counters;  // acc pairs, grad pairs, tstep pairs, hhs calls, fsi calls, max depth
    unsigned long long *levels;    // [2][SUBTREE_STAT_LEVELS]: calls and set sizes per depth
};

struct SubWork {
    int32_t *perm, *tmp;
    double *tau;
    double *aA, *aB, *atA, *atB;  // [3][n] each
    float *wA, *wB;
    float4 *recA, *recB;          // 64 bytes per particle each
};

struct Counts {
    unsigned long long acc, grad, tstep, hhs, fsi;
    int maxdepth;
};

// ---- block-level building blocks ----------------------------------------------------

template <bool MIXED>
__device__ void b_pack_pos(const SubParams &p, const int32_t *L, int n, void *rec, bool accurate)
{
    for (int k = threadIdx.x; k < n; k += SB) {
        if (MIXED) {
            if (accurate) pack_grad_mixed_one(k, L, n, p.x, p.m, p.N, nullptr, (float4 *)rec);
            else pack_pos_mixed_one(k, L, n, p.x, p.m, p.N, (float4 *)rec);
        } else {
            pack_pos_fp64_one(k, L, n, p.x, p.m, p.N, (double4_32a *)rec);
        }
    }
}

// Newtonian pass of A against B (self: the same list): out[3][nA] = G sum; wout[nA] =
// max_j m_j / r^3 when the accurate variant runs (mixed mode, before a gradient pass)
template <bool MIXED>
__device__ __noinline__ void b_acc(const SubParams &p, const SubWork &w, const int32_t *A, int nA, const int32_t *B,
                      int nB, bool self, bool accurate, double *out, float *wout, Counts &cnt)
{
    if (nA <= 0) return;
    const int badbit = p.eps2 == 0.0 ? ERR_COINCIDENT : ERR_NONFINITE;
    if (nB <= 0 || (self && nA == 1)) {
        for (int k = threadIdx.x; k < nA; k += SB) {
            out[k] = out[nA + k] = out[2 * nA + k] = 0.0;
            if (wout) wout[k] = 0.f;
        }
        __syncthreads();
        return;
    }
    accurate = accurate && MIXED;
    b_pack_pos<MIXED>(p, A, nA, w.recA, accurate);
    if (!self) b_pack_pos<MIXED>(p, B, nB, w.recB, accurate);
    __syncthreads();
    const int sp = self ? 1 : 0;
    if (MIXED) {
        const float4 *ir = w.recA, *jr = self ? w.recA : w.recB;
        for (int ib = 0; ib < nA; ib += SIB) {
            double res[SILP][3];
            float wr[SILP];
            if (accurate) acc3_mixed_body<SB, SILP, STJ>(ir, jr, nA, nB, ib, 0, nB, sp, (float)p.eps2, res, wr);
            else acc_mixed_body<SB, SILP, STJ, false>(ir, jr, nA, nB, ib, 0, nB, sp, (float)p.eps2, res, wr);
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                const int i = ib + k * SB + threadIdx.x;
                if (i < nA) {
                    bool ok = true;
                    for (int c = 0; c < 3; ++c) {
                        const double a = p.G * res[k][c];
                        ok = ok && isfinite(a);
                        out[c * nA + i] = a;
                    }
                    if (wout) wout[i] = wr[k];
                    if (!ok) atomicOr(p.err, badbit);
                }
            }
        }
    } else {
        const double4_32a *ir = (const double4_32a *)w.recA;
        const double4_32a *jr = self ? ir : (const double4_32a *)w.recB;
        for (int ib = 0; ib < nA; ib += SB) {
            double res[3];
            acc_fp64_body<SB, STJ>(ir, jr, nA, nB, ib, 0, nB, sp, p.eps2, res);
            const int i = ib + threadIdx.x;
            if (i < nA) {
                bool ok = true;
                for (int c = 0; c < 3; ++c) {
                    const double a = p.G * res[c];
                    ok = ok && isfinite(a);
                    out[c * nA + i] = a;
                }
                if (!ok) atomicOr(p.err, badbit);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cnt.acc += self ? (unsigned long long)nA * (nA - 1) : (unsigned long long)nA * nB;
}

// Gradient pass of A against B with a_A, a_B ([3][n]); at[3][nA] = a_A + eps^2/48 g
template <bool MIXED>
__device__ __noinline__ void b_grad(const SubParams &p, const SubWork &w, const int32_t *A, int nA, const double *aA,
                       const int32_t *B, int nB, const double *aB, bool self, double eps_grad,
                       const float *wmax, double *at, Counts &cnt)
{
    if (nA <= 0) return;
    const int badbit = p.eps2 == 0.0 ? ERR_COINCIDENT : ERR_NONFINITE;
    if (nB <= 0 || (self && nA == 1)) {
        for (int k = threadIdx.x; k < 3 * nA; k += SB) at[k] = aA[k];
        __syncthreads();
        return;
    }
    for (int k = threadIdx.x; k < nA; k += SB) {
        if (MIXED) pack_grad_mixed_one(k, A, nA, p.x, p.m, p.N, aA, w.recA);
        else pack_grad_fp64_one(k, A, nA, p.x, p.m, p.N, aA, (double4_32a *)w.recA);
    }
    if (!self)
        for (int k = threadIdx.x; k < nB; k += SB) {
            if (MIXED) pack_grad_mixed_one(k, B, nB, p.x, p.m, p.N, aB, w.recB);
            else pack_grad_fp64_one(k, B, nB, p.x, p.m, p.N, aB, (double4_32a *)w.recB);
        }
    __syncthreads();
    const int sp = self ? 1 : 0;
    const double c = eps_grad * eps_grad / 48.0;
    const double scale = 2.0 * p.G;
    if (MIXED) {
        const float4 *ir = w.recA, *jr = self ? w.recA : w.recB;
        for (int ib = 0; ib < nA; ib += SIB) {
            double res[SILP][3];
            grad_mixed_body<SB, SILP, STJ>(ir, jr, nA, nB, ib, 0, nB, sp, p.eps2, wmax, res);
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                const int i = ib + k * SB + threadIdx.x;
                if (i < nA) {
                    bool ok = true;
                    for (int q = 0; q < 3; ++q) {
                        const double v = aA[q * nA + i] + c * (scale * res[k][q]);
                        ok = ok && isfinite(v);
                        at[q * nA + i] = v;
                    }
                    if (!ok) atomicOr(p.err, badbit);
                }
            }
        }
    } else {
        const double4_32a *ir = (const double4_32a *)w.recA;
        const double4_32a *jr = self ? ir : (const double4_32a *)w.recB;
        for (int ib = 0; ib < nA; ib += SB) {
            double res[3];
            grad_fp64_body<SB, STJ>(ir, jr, nA, nB, ib, 0, nB, sp, p.eps2, res);
            const int i = ib + threadIdx.x;
            if (i < nA) {
                bool ok = true;
                for (int q = 0; q < 3; ++q) {
                    const double v = aA[q * nA + i] + c * (scale * res[q]);
                    ok = ok && isfinite(v);
                    at[q * nA + i] = v;
                }
                if (!ok) atomicOr(p.err, badbit);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cnt.grad += self ? (unsigned long long)nA * (nA - 1) : (unsigned long long)nA * nB;
}

// symmetrised time-steps of the set P into tau[n]
template <bool MIXED, int SYM>
__device__ __noinline__ void b_tstep(const SubParams &p, const SubWork &w, const int32_t *P, int n, double *tau, Counts &cnt)
{
    if (n <= 0) return;
    if (n == 1) {
        if (threadIdx.x == 0) tau[0] = INFINITY;
        __syncthreads();
        return;
    }
    for (int k = threadIdx.x; k < n; k += SB) {
        if (MIXED) pack_tstep_mixed_one(k, P, n, p.x, p.v, p.m, p.N, p.G, w.recA);
        else pack_tstep_fp64_one(k, P, n, p.x, p.v, p.m, p.N, p.G, (double4_32a *)w.recA);
    }
    __syncthreads();
    if (MIXED) {
        for (int ib = 0; ib < n; ib += SIB) {
            float best[SILP], minr2[SILP];
            tstep_mixed_body<SB, SILP, STJ, SYM>(w.recA, w.recA, n, n, ib, 0, n, 1, (float)p.eta, best, minr2);
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                const int i = ib + k * SB + threadIdx.x;
                if (i < n) {
                    const double t = p.eta * (double)best[k];
                    tau[i] = t;
                    if (minr2[k] == 0.f) atomicOr(p.err, ERR_COINCIDENT);
                    if (!(t > 0.0)) atomicOr(p.err, ERR_NONFINITE);
                }
            }
        }
    } else {
        const double4_32a *r = (const double4_32a *)w.recA;
        for (int ib = 0; ib < n; ib += SB) {
            double best, minr2;
            tstep_fp64_body<SB, STJ, SYM>(r, r, n, n, ib, 0, n, 1, p.eta, best, minr2);
            const int i = ib + threadIdx.x;
            if (i < n) {
                const double t = p.eta * best;
                tau[i] = t;
                if (minr2 == 0.0) atomicOr(p.err, ERR_COINCIDENT);
                if (!(t > 0.0)) atomicOr(p.err, ERR_NONFINITE);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cnt.tstep += (unsigned long long)n * (n - 1);
}

// stable in-place partition of P[0..n) by tau >= pivot; returns |S| (S first, then F)
__device__ __noinline__ int b_partition(int32_t *P, int n, const double *tau, double pivot, int32_t *tmp)
{
    __shared__ int wsum[SB / 32];
    __shared__ int s_chunk, s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // slow count
    int c = 0;
    for (int k = tid; k < n; k += SB) c += (tau[k] >= pivot) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) wsum[warp] = c;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int q = 0; q < SB / 32; ++q) t += wsum[q];
        s_total = t;
    }
    __syncthreads();
    const int nS = s_total;
    int sbase = 0, fbase = 0;
    for (int c0 = 0; c0 < n; c0 += SB) {
        const int k = c0 + tid;
        const bool valid = k < n;
        const bool slow = valid && (tau[k] >= pivot);
        const unsigned bal = __ballot_sync(0xffffffffu, slow);
        const int rank = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int q = 0; q < SB / 32; ++q) {
                const int v = wsum[q];
                wsum[q] = t;
                t += v;
            }
            s_chunk = t;
        }
        __syncthreads();
        if (valid) {
            const int before = wsum[warp] + rank;  // slow entries before k in this chunk
            if (slow) tmp[sbase + before] = P[k];
            else tmp[nS + fbase + (tid - before)] = P[k];
        }
        const int tot = s_chunk;
        sbase += tot;
        fbase += min(SB, n - c0) - tot;
        __syncthreads();
    }
    for (int k = tid; k < n; k += SB) P[k] = tmp[k];
    __syncthreads();
    return nS;
}

__device__ void b_kick(const SubParams &p, const int32_t *L, int n, const double *a, double dt)
{
    for (int k = threadIdx.x; k < n; k += SB) {
        const int i = L[k];
        for (int c = 0; c < 3; ++c)
            p.v[c * p.N + i] = __dadd_rn(p.v[c * p.N + i], __dmul_rn(dt, a[c * n + k]));
    }
    __syncthreads();
}

__device__ void b_drift(const SubParams &p, const int32_t *L, int n, double dt)
{
    for (int k = threadIdx.x; k < n; k += SB) {
        const int i = L[k];
        for (int c = 0; c < 3; ++c)
            p.x[c * p.N + i] = __dadd_rn(p.x[c * p.N + i], __dmul_rn(dt, p.v[c * p.N + i]));
    }
    __syncthreads();
}

// Algorithm fsi on the set S with step dt
template <bool MIXED>
__device__ __noinline__ void b_fsi(const SubParams &p, const SubWork &w, const int32_t *S, int nS, double dt, Counts &cnt)
{
    if (nS <= 0) return;
    if (threadIdx.x == 0) cnt.fsi += 1;
    b_acc<MIXED>(p, w, S, nS, S, nS, true, false, w.aA, nullptr, cnt);
    b_kick(p, S, nS, w.aA, dt / 6.0);
    b_drift(p, S, nS, 0.5 * dt);
    b_acc<MIXED>(p, w, S, nS, S, nS, true, true, w.aA, w.wA, cnt);
    b_grad<MIXED>(p, w, S, nS, w.aA, S, nS, w.aA, true, dt, MIXED ? w.wA : nullptr, w.atA, cnt);
    b_kick(p, S, nS, w.atA, 2.0 * dt / 3.0);
    b_drift(p, S, nS, 0.5 * dt);
    b_acc<MIXED>(p, w, S, nS, S, nS, true, false, w.aA, nullptr, cnt);
    b_kick(p, S, nS, w.aA, dt / 6.0);
}

// kick_sf: S kicked by its accelerations due to F, F by those due to S (computed first)
template <bool MIXED>
__device__ __noinline__ void b_kick_sf(const SubParams &p, const SubWork &w, const int32_t *S, int nS, const int32_t *F,
                          int nF, double cdt, bool gradient, double tau, Counts &cnt)
{
    if (nS <= 0 || nF <= 0) return;
    b_acc<MIXED>(p, w, S, nS, F, nF, false, gradient, w.aA, gradient ? w.wA : nullptr, cnt);
    b_acc<MIXED>(p, w, F, nF, S, nS, false, gradient, w.aB, gradient ? w.wB : nullptr, cnt);
    if (gradient) {
        b_grad<MIXED>(p, w, S, nS, w.aA, F, nF, w.aB, false, tau, MIXED ? w.wA : nullptr, w.atA, cnt);
        b_grad<MIXED>(p, w, F, nF, w.aB, S, nS, w.aA, false, tau, MIXED ? w.wB : nullptr, w.atB, cnt);
        b_kick(p, S, nS, w.atA, cdt);
        b_kick(p, F, nF, w.atB, cdt);
    } else {
        b_kick(p, S, nS, w.aA, cdt);
        b_kick(p, F, nF, w.aB, cdt);
    }
}

// One block: n_steps calls of hhs_fsi(P, tau0) at depth depth0.  Single-set mode: P, n given,
// workspace from particle 0.  Batch mode (offsets != NULL): block b takes the particles
// [offsets[b], offsets[b+1]) in order, and the workspace region of those particles.
template <bool MIXED, int SYM>
__global__ void __launch_bounds__(SB) k_hhs_subtree(SubParams p, SubWork w0, const int32_t *__restrict__ P,
                                                    int n_single, const int64_t *__restrict__ offsets,
                                                    double tau0, int depth0, int n_steps)
{
    __shared__ int f_lo[MAXD], f_n[MAXD], f_ns[MAXD], f_pc[MAXD], f_depth[MAXD];
    __shared__ double f_tau[MAXD];
    __shared__ int s_sp, s_abort;
    const int tid = threadIdx.x;
    int off = 0, n = n_single;
    if (offsets) {
        off = (int)offsets[blockIdx.x];
        n = (int)(offsets[blockIdx.x + 1] - offsets[blockIdx.x]);
    }
    SubWork w = w0;
    w.perm += off;
    w.tmp += off;
    w.tau += off;
    w.aA += 3 * (size_t)off;
    w.aB += 3 * (size_t)off;
    w.atA += 3 * (size_t)off;
    w.atB += 3 * (size_t)off;
    w.wA += off;
    w.wB += off;
    w.recA += 4 * (size_t)off;
    w.recB += 4 * (size_t)off;
    Counts cnt = {0, 0, 0, 0, 0, depth0};
    if (tid == 0) s_abort = 0;
    for (int step = 0; step < n_steps; ++step) {
        for (int k = tid; k < n; k += SB) w.perm[k] = offsets ? off + k : P[k];
        if (tid == 0) {
            s_sp = 1;
            f_lo[0] = 0;
            f_n[0] = n;
            f_ns[0] = 0;
            f_pc[0] = 0;
            f_depth[0] = depth0;
            f_tau[0] = tau0;
        }
        __syncthreads();
        while (true) {
            if (s_sp == 0 || s_abort) break;
            const int top = s_sp - 1;
            const int lo = f_lo[top], fn = f_n[top], pc = f_pc[top], depth = f_depth[top];
            const double ftau = f_tau[top];
            int nS = f_ns[top];
            __syncthreads();  // every thread has read the frame before it changes
            int32_t *S = w.perm + lo;
            if (pc == 0) {
                if (depth > p.max_depth) {
                    if (tid == 0) {
                        atomicOr(p.err, ERR_DEPTH);
                        s_abort = 1;
                    }
                    __syncthreads();
                    break;
                }
                if (tid == 0) {
                    cnt.hhs += 1;
                    cnt.maxdepth = max(cnt.maxdepth, depth);
                    const int L = min(depth, SUBTREE_STAT_LEVELS - 1);
                    atomicAdd(&p.levels[L], 1ull);
                    atomicAdd(&p.levels[SUBTREE_STAT_LEVELS + L], (unsigned long long)fn);
                }
                b_tstep<MIXED, SYM>(p, w, S, fn, w.tau, cnt);
                nS = b_partition(S, fn, w.tau, ftau, w.tmp);
                const int nF = fn - nS;
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, ftau / 6.0, false, ftau, cnt);
                b_fsi<MIXED>(p, w, S, nS, 0.5 * ftau, cnt);
                if (tid == 0) {
                    f_ns[top] = nS;
                    f_pc[top] = 1;
                    if (nF > 0) {
                        if (s_sp >= MAXD) {
                            atomicOr(p.err, ERR_DEPTH);
                            s_abort = 1;
                        } else {
                            f_lo[s_sp] = lo + nS;
                            f_n[s_sp] = nF;
                            f_ns[s_sp] = 0;
                            f_pc[s_sp] = 0;
                            f_depth[s_sp] = depth + 1;
                            f_tau[s_sp] = 0.5 * ftau;
                            s_sp += 1;
                        }
                    }
                }
            } else if (pc == 1) {
                const int nF = fn - nS;
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, 2.0 * ftau / 3.0, true, ftau, cnt);
                if (tid == 0) {
                    f_pc[top] = 2;
                    if (nF > 0) {
                        f_lo[s_sp] = lo + nS;
                        f_n[s_sp] = nF;
                        f_ns[s_sp] = 0;
                        f_pc[s_sp] = 0;
                        f_depth[s_sp] = depth + 1;
                        f_tau[s_sp] = 0.5 * ftau;
                        s_sp += 1;
                    }
                }
            } else {
                const int nF = fn - nS;
                b_fsi<MIXED>(p, w, S, nS, 0.5 * ftau, cnt);
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, ftau / 6.0, false, ftau, cnt);
                if (tid == 0) s_sp -= 1;
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_abort) break;
    }
    if (tid == 0) {
        atomicAdd(&p.counters[0], cnt.acc);
        atomicAdd(&p.counters[1], cnt.grad);
        atomicAdd(&p.counters[2], cnt.tstep);
        atomicAdd(&p.counters[3], cnt.hhs);
        atomicAdd(&p.counters[4], cnt.fsi);
        atomicMax(&p.counters[5], (unsigned long long)cnt.maxdepth);
    }
}

}  // namespace

void launch_subtree(cudaStream_t s, bool mixed, int sym, const SubtreeArgs &a)
{
    SubParams p;
    p.x = a.x;
    p.v = a.v;
    p.m = a.m;
    p.N = a.N;
    p.G = a.G;
    p.eta = a.eta;
    p.eps2 = a.eps2;
    p.max_depth = a.max_depth;
    p.err = a.err;
    p.counters = a.counters;
    p.levels = a.levels;
    SubWork w;
    w.perm = a.perm;
    w.tmp = a.tmp;
    w.tau = a.tau;
    w.aA = a.aA;
    w.aB = a.aB;
    w.atA = a.atA;
    w.atB = a.atB;
    w.wA = a.wA;
    w.wB = a.wB;
    w.recA = (float4 *)a.recA;
    w.recB = (float4 *)a.recB;
    const unsigned nblk = a.offsets ? (unsigned)a.n_blocks : 1u;
#define FROST_SUBTREE_CASE(MIX, SYMV)                                                             \
    k_hhs_subtree<MIX, SYMV><<<nblk, SB, 0, s>>>(p, w, a.P, a.n, a.offsets, a.tau0, a.depth0, a.n_steps)
    if (mixed) {
        if (sym == 0) FROST_SUBTREE_CASE(true, 0);
        else if (sym == 1) FROST_SUBTREE_CASE(true, 1);
        else FROST_SUBTREE_CASE(true, 2);
    } else {
        if (sym == 0) FROST_SUBTREE_CASE(false, 0);
        else if (sym == 1) FROST_SUBTREE_CASE(false, 1);
        else FROST_SUBTREE_CASE(false, 2);
    }
#undef FROST_SUBTREE_CASE
}

}  // namespace frost
