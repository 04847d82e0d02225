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

// The coefficients of one step h of the FSI and of kick_sf: h, h/6, 2h/3 and h^2/48.  A level's
// pivot step is exactly half its parent's, and rounding commutes with scaling by a power of
// two, so the coefficients of every level are exact powers-of-two multiples of those of the
// launch's first step: a table of them per launch gives the bits of the divisions without the
// divisions (an FP64 division is a sequence of FP64 instructions, each of which holds a
// sub-partition's FP64 unit for about 64 cycles).
struct StepK {
    double h, k6, k23, k48;
};

struct SubParams {
    double *x, *v;
    const double *m;
    int N;
    double G, eta, eps2;
    int max_depth;
    int *err;
    unsigned long long *counters;  // acc pairs, grad pairs, tstep pairs, hhs calls, fsi calls, max depth
    unsigned long long *levels;    // [2][SUBTREE_STAT_LEVELS]: calls and set sizes per depth
    int crank, csize;              // this block's rank in its thread-block cluster, cluster size
    double *aC;                    // [3][N] by particle: a^SS kept between the two fsi(S) of a call
    // the team's threads within each block: tbase .. tbase + tcount - 1 (the whole block, or
    // warps 1..7 of a one-block team while warp 0 runs a fast set's subtree beside them)
    int tbase, tcount;
    int overlap;                   // run fsi(S) beside the warp path of F (one-block teams)
    const StepK *K;                // shared: K[r] for the step tau0 2^-r, r = 0..MAXD
    int kdepth0;                   // the depth of tau0
};

struct SubWork {
    int *xchg;                    // one int per cluster of blocks: the warp path's status
    int32_t *perm, *tmp;
    double *tau;
    double *aA, *aB, *atA, *atB;  // [3][n] each
    float *wA, *wB;
    float4 *recA, *recB;          // 64 bytes per particle each
};

struct Counts {
    unsigned long long acc, grad, tstep, hhs, fsi;
    int maxdepth;
    unsigned long long reused;
    unsigned long long beside;  // fsi(S) steps run on warps 1..7 beside the warp path of F
};

// ---- the team of one set: a block, or the blocks of a thread-block cluster -----------------
// Every helper below is called by all threads of the team with the same arguments, splits its
// work over the team's threads and ends with a team barrier, so that all control decisions,
// taken from data read after a barrier, are the same in every block of a cluster.  A one-block
// team may also be the sub-team of warps 1..7 (tbase 32, tcount 224), which runs the FSI steps
// of a slow set while warp 0 advances the fast set; its barrier is the named barrier 1.

constexpr int SUB_BARRIER = 1;    // named barrier of the warps 1..7 sub-team (0 is __syncthreads)

// G times a sum; G = 1 (Henon units) needs no FP64 multiply and gives the same bits
__device__ __forceinline__ double g_scale(double G, double r) { return G == 1.0 ? r : G * r; }

__device__ __forceinline__ int t_id(const SubParams &p) { return p.crank * p.tcount + ((int)threadIdx.x - p.tbase); }
__device__ __forceinline__ int t_n(const SubParams &p) { return p.csize * p.tcount; }
__device__ __forceinline__ bool t_lead(const SubParams &p) { return (int)threadIdx.x == p.tbase; }

// team barrier: with more than one block, the cluster barrier (release / acquire at cluster
// scope orders the global-memory results of every block before the next step); a sub-team
// waits at its named barrier, which orders memory among its threads as __syncthreads does
__device__ __forceinline__ void t_sync(const SubParams &p)
{
    if (p.csize > 1) {
        asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    } else if (p.tcount != SB) {
        asm volatile("bar.sync %0, %1;" ::"n"(SUB_BARRIER), "r"(p.tcount) : "memory");
    } else {
        __syncthreads();
    }
}

// ---- block-level building blocks ----------------------------------------------------

template <bool MIXED>
__device__ void b_pack_pos(const SubParams &p, const int32_t *L, int n, void *rec)
{
    for (int k = t_id(p); k < n; k += t_n(p)) {
        if (MIXED) {
            pack_pos_mixed_one(k, L, n, p.x, p.m, p.N, (float4 *)rec);
        } else {
            pack_pos_fp64_one(k, L, n, p.x, p.m, p.N, (double4_32a *)rec);
        }
    }
}

// ---- several threads per active particle (sets of at most MT_MAX) ----------------------
// For a small active list the one-thread-per-particle bodies leave most of the block idle and
// run long dependent j-loops.  Here T = SB / pow2ceil(nA) threads (a power of two, at most 32,
// adjacent lanes of one warp) share particle i = tid / T: lane l of the group takes the
// sources l, l + T, l + 2T, ... and the group sums its partials with a butterfly of shuffles,
// which fixes the order (deterministic).  Every thread runs the same number of j-iterations
// (out-of-range sources are masked as the self pair), as the time-step pairs vote per warp.
constexpr int MT_MAX = SB;

// lanes per particle T (a power of two, at most 32) over the team's threads, group g and lane
// l of this thread, and the rounds over the particles when they outnumber the groups
struct MtMap {
    int T, g, l, ngroups, rounds;
};
// T depends on the size of the whole team (csize blocks of SB threads), not on that of a
// sub-team, so a pass gives the same bits on either; a sub-team takes more rounds instead
__device__ __forceinline__ MtMap mt_map(const SubParams &p, int nA)
{
    int P2 = 1;
    while (P2 < nA) P2 <<= 1;
    MtMap m;
    m.T = max(1, min(32, p.csize * SB / P2));
    m.g = t_id(p) / m.T;
    m.l = t_id(p) % m.T;
    m.ngroups = t_n(p) / m.T;
    m.rounds = (nA + m.ngroups - 1) / m.ngroups;
    return m;
}

__device__ __forceinline__ double grp_sum(double v, int T)
{
    for (int o = T >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float grp_max(float v, int T)
{
    for (int o = T >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float grp_min(float v, int T)
{
    for (int o = T >> 1; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double grp_mind(double v, int T)
{
    for (int o = T >> 1; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// source index and masking position of iteration q for lane l: sources past the end repeat the
// last one and are masked as the self pair (jpos == ipos); in a cross pass jpos = -1 otherwise
struct MtSrc {
    int j, jpos;
};
__device__ __forceinline__ MtSrc mt_src(int q, int T, int l, int nB, int i, bool self)
{
    const int j0 = q * T + l;
    const bool valid = j0 < nB;
    MtSrc r;
    r.j = valid ? j0 : nB - 1;
    r.jpos = valid ? (self ? j0 : -1) : i;
    return r;
}

// Newtonian pass (records as in b_acc); out / wout written by lane 0 of each group
template <bool MIXED>
__device__ __noinline__ void mt_acc(const SubParams &p, const void *irec, const void *jrec, int nA, int nB, bool self,
                                    bool accurate, double *out, float *wout, int badbit)
{
    const MtMap mm = mt_map(p, nA);
    const int T = mm.T, l = mm.l;
    const int nq = (nB + T - 1) / T;
    for (int rr = 0; rr < mm.rounds; ++rr) {
        const int i0 = mm.g + rr * mm.ngroups;
        const bool active = i0 < nA;
        const int i = active ? i0 : 0;
        const int ipos[1] = {i};
        double r[3];
        float wm[1] = {0.f};
        if (MIXED) {
            const float4 *ir = (const float4 *)irec, *jr = (const float4 *)jrec;
            const float eps2 = (float)p.eps2;
            float H[3] = {0.f, 0.f, 0.f}, L[3] = {0.f, 0.f, 0.f};
            float ax[1] = {0.f}, ay[1] = {0.f}, az[1] = {0.f};
            int c = 0;
            AccMixedI<1> I;
            const float4 q0 = ir[i], q1 = ir[nA + i];
            I.xh[0] = q0.x; I.yh[0] = q0.y; I.zh[0] = q0.z;
            I.xl[0] = q1.x; I.yl[0] = q1.y; I.zl[0] = q1.z;
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, nB, i, self);
                if (accurate)
                    acc_mixed_j<1, true, true, true>(jr[s.j], jr[nB + s.j], I, eps2, s.jpos, ipos, ax, ay, az, wm);
                else
                    acc_mixed_j<1, true, false>(jr[s.j], jr[nB + s.j], I, eps2, s.jpos, ipos, ax, ay, az, wm);
                if (++c == 16) {
                    fold2(H[0], L[0], ax[0]); fold2(H[1], L[1], ay[0]); fold2(H[2], L[2], az[0]);
                    ax[0] = ay[0] = az[0] = 0.f;
                    c = 0;
                }
            }
            fold2(H[0], L[0], ax[0]); fold2(H[1], L[1], ay[0]); fold2(H[2], L[2], az[0]);
            for (int k = 0; k < 3; ++k) r[k] = (double)H[k] + (double)L[k];
        } else {
            const double4_32a *ir = (const double4_32a *)irec, *jr = (const double4_32a *)jrec;
            const double4_32a I = ir[i];
            r[0] = r[1] = r[2] = 0.0;
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, nB, i, self);
                acc_fp64_j<true>(jr[s.j], I, p.eps2, s.jpos, i, r[0], r[1], r[2]);
            }
        }
        for (int k = 0; k < 3; ++k) r[k] = grp_sum(r[k], T);
        const float wmx = grp_max(wm[0], T);
        if (active && l == 0) {
            bool ok = true;
            for (int k = 0; k < 3; ++k) {
                const double a = g_scale(p.G, r[k]);
                ok = ok && isfinite(a);
                out[k * nA + i] = a;
            }
            if (wout) wout[i] = wmx;
            if (!ok) atomicOr(p.err, badbit);
        }
    }
}

// gradient pass (records as in b_grad): at[3][nA] = a_A + c 2G sum
template <bool MIXED>
__device__ __noinline__ void mt_grad(const SubParams &p, const void *irec, const void *jrec, int nA, int nB, bool self,
                                     const double *aA, const float *wmax, double c, double *at, int badbit)
{
    const MtMap mm = mt_map(p, nA);
    const int T = mm.T, l = mm.l;
    const int nq = (nB + T - 1) / T;
    for (int rr = 0; rr < mm.rounds; ++rr) {
        const int i0 = mm.g + rr * mm.ngroups;
        const bool active = i0 < nA;
        const int i = active ? i0 : 0;
        const int ipos[1] = {i};
        double r[3];
        if (MIXED) {
            const float4 *ir = (const float4 *)irec, *jr = (const float4 *)jrec;
            const float eps2 = (float)p.eps2;
            GradMixedI<1> I;
            const float4 q0 = ir[i], q1 = ir[nA + i], q2 = ir[2 * nA + i], q3 = ir[3 * nA + i];
            I.xh[0] = q0.x; I.yh[0] = q0.y; I.zh[0] = q0.z;
            I.xm[0] = q1.x; I.ym[0] = q1.y; I.zm[0] = q1.z; I.ahx[0] = q1.w;
            I.xl[0] = q2.x; I.yl[0] = q2.y; I.zl[0] = q2.z; I.ahy[0] = q2.w;
            I.ahz[0] = q3.x; I.alx[0] = q3.y; I.aly[0] = q3.z; I.alz[0] = q3.w;
            const float thr[1] = {wmax ? SLOT_FRACTION * wmax[i] : INFINITY};
            BigSlots<1> big;
            init_big(big, 0);
            float H[3] = {0.f, 0.f, 0.f}, L[3] = {0.f, 0.f, 0.f};
            float gx[1] = {0.f}, gy[1] = {0.f}, gz[1] = {0.f};
            int cnt = 0;
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, nB, i, self);
                grad_mixed_j<1, true>(jr[s.j], jr[nB + s.j], jr[2 * nB + s.j], jr[3 * nB + s.j], I, eps2, s.j, s.jpos,
                                      ipos, thr, big, gx, gy, gz);
                if (++cnt == 16) {
                    fold2(H[0], L[0], gx[0]); fold2(H[1], L[1], gy[0]); fold2(H[2], L[2], gz[0]);
                    gx[0] = gy[0] = gz[0] = 0.f;
                    cnt = 0;
                }
            }
            fold2(H[0], L[0], gx[0]); fold2(H[1], L[1], gy[0]); fold2(H[2], L[2], gz[0]);
            double bx = 0.0, by = 0.0, bz = 0.0;
#pragma unroll
            for (int t = 0; t < GRAD_SLOTS; ++t) {
                if (t < big.n[0]) {
                    const int j = big.j[t][0];
                    grad_term_df<1>(jr[j], jr[nB + j], jr[2 * nB + j], jr[3 * nB + j], I, 0, p.eps2, bx, by, bz);
                }
            }
            r[0] = ((double)H[0] + (double)L[0]) + bx;
            r[1] = ((double)H[1] + (double)L[1]) + by;
            r[2] = ((double)H[2] + (double)L[2]) + bz;
        } else {
            const double4_32a *ir = (const double4_32a *)irec, *jr = (const double4_32a *)jrec;
            const double4_32a I = ir[i], IA = ir[nA + i];
            r[0] = r[1] = r[2] = 0.0;
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, nB, i, self);
                grad_fp64_j<true>(jr[s.j], jr[nB + s.j], I, IA, p.eps2, s.jpos, i, r[0], r[1], r[2]);
            }
        }
        for (int k = 0; k < 3; ++k) r[k] = grp_sum(r[k], T);
        if (active && l == 0) {
            bool ok = true;
            for (int k = 0; k < 3; ++k) {
                const double v = aA[k * nA + i] + c * (2.0 * p.G * r[k]);
                ok = ok && isfinite(v);
                at[k * nA + i] = v;
            }
            if (!ok) atomicOr(p.err, badbit);
        }
    }
}

// time-step pass of the set (records as in b_tstep): tau[i] = eta min_j (...)
template <bool MIXED, int SYM>
__device__ __noinline__ void mt_tstep(const SubParams &p, const void *rec, int n, double *tau)
{
    const MtMap mm = mt_map(p, n);
    const int T = mm.T, l = mm.l;
    const int nq = (n + T - 1) / T;
    for (int rr = 0; rr < mm.rounds; ++rr) {
        const int i0 = mm.g + rr * mm.ngroups;
        const bool active = i0 < n;
        const int i = active ? i0 : 0;
        const int ipos[1] = {i};
        double t;
        bool coincident;
        if (MIXED) {
            const float4 *r = (const float4 *)rec;
            TstepMixedI<1> I;
            const float4 a = r[i], b = r[n + i], cc = r[2 * n + i];
            const float4 da = (SYM & 4) ? r[3 * n + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            I.xh[0] = a.x; I.yh[0] = a.y; I.zh[0] = a.z;
            I.xl[0] = b.x; I.yl[0] = b.y; I.zl[0] = b.z;
            I.vx[0] = cc.x; I.vy[0] = cc.y; I.vz[0] = cc.z; I.gm[0] = cc.w;
            I.ax[0] = da.x; I.ay[0] = da.y; I.az[0] = da.z;
            const float eta = (float)p.eta, eta15 = 1.5f * eta;
            float best[1] = {INFINITY}, minr2[1] = {INFINITY};
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, n, i, true);
                const float4 JA = (SYM & 4) ? r[3 * n + s.j] : make_float4(0.f, 0.f, 0.f, 0.f);
                tstep_mixed_j<1, SYM, true>(r[s.j], r[n + s.j], r[2 * n + s.j], JA, I, eta, eta15, s.jpos, ipos,
                                            best, minr2);
            }
            t = p.eta * (double)grp_min(best[0], T);
            coincident = grp_min(minr2[0], T) == 0.f;
        } else {
            const double4_32a *r = (const double4_32a *)rec;
            const double4_32a zero4 = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            const double4_32a I = r[i], IV = r[n + i], IA = (SYM & 4) ? r[2 * n + i] : zero4;
            double best = INFINITY, minr2 = INFINITY;
            for (int q = 0; q < nq; ++q) {
                const MtSrc s = mt_src(q, T, l, n, i, true);
                tstep_fp64_j<SYM, true>(r[s.j], r[n + s.j], (SYM & 4) ? r[2 * n + s.j] : zero4, I, IV, IA, p.eta,
                                        s.jpos, i, best, minr2);
            }
            t = p.eta * grp_mind(best, T);
            coincident = grp_mind(minr2, T) == 0.0;
        }
        if (active && l == 0) {
            tau[i] = t;
            if (coincident) atomicOr(p.err, ERR_COINCIDENT);
            if (!(t > 0.0)) atomicOr(p.err, ERR_NONFINITE);
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
        for (int k = t_id(p); k < nA; k += t_n(p)) {
            out[k] = out[nA + k] = out[2 * nA + k] = 0.0;
            if (wout) wout[k] = 0.f;
        }
        t_sync(p);
        return;
    }
    accurate = accurate && MIXED;
    b_pack_pos<MIXED>(p, A, nA, w.recA);
    if (!self) b_pack_pos<MIXED>(p, B, nB, w.recB);
    t_sync(p);
    const int sp = self ? 1 : 0;
    if (p.csize > 1 || nA <= MT_MAX || p.tcount != SB) {
        mt_acc<MIXED>(p, w.recA, self ? w.recA : w.recB, nA, nB, self, accurate, out, wout, badbit);
    } else if (MIXED) {
        const float4 *ir = w.recA, *jr = self ? w.recA : w.recB;
        for (int ib = 0; ib < nA; ib += SIB) {
            double res[SILP][3];
            float wr[SILP];
            if (accurate) acc_mixed_body<SB, SILP, STJ, true, true>(ir, jr, nA, nB, ib, 0, nB, sp, (float)p.eps2, res, wr);
            else acc_mixed_body<SB, SILP, STJ, false>(ir, jr, nA, nB, ib, 0, nB, sp, (float)p.eps2, res, wr);
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                const int i = ib + k * SB + threadIdx.x;
                if (i < nA) {
                    bool ok = true;
                    for (int c = 0; c < 3; ++c) {
                        const double a = g_scale(p.G, res[k][c]);
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
                    const double a = g_scale(p.G, res[c]);
                    ok = ok && isfinite(a);
                    out[c * nA + i] = a;
                }
                if (!ok) atomicOr(p.err, badbit);
            }
        }
    }
    t_sync(p);
    if (t_lead(p)) cnt.acc += self ? (unsigned long long)nA * (nA - 1) : (unsigned long long)nA * nB;
}

// Gradient pass of A against B with a_A, a_B ([3][n]); at[3][nA] = a_A + c48 g, c48 = eps^2/48
template <bool MIXED>
__device__ __noinline__ void b_grad(const SubParams &p, const SubWork &w, const int32_t *A, int nA, const double *aA,
                       const int32_t *B, int nB, const double *aB, bool self, double c48,
                       const float *wmax, double *at, Counts &cnt)
{
    if (nA <= 0) return;
    const int badbit = p.eps2 == 0.0 ? ERR_COINCIDENT : ERR_NONFINITE;
    if (nB <= 0 || (self && nA == 1)) {
        for (int k = t_id(p); k < 3 * nA; k += t_n(p)) at[k] = aA[k];
        t_sync(p);
        return;
    }
    for (int k = t_id(p); k < nA; k += t_n(p)) {
        if (MIXED) pack_grad_mixed_one(k, A, nA, p.x, p.m, p.N, aA, w.recA);
        else pack_grad_fp64_one(k, A, nA, p.x, p.m, p.N, aA, (double4_32a *)w.recA);
    }
    if (!self)
        for (int k = t_id(p); k < nB; k += t_n(p)) {
            if (MIXED) pack_grad_mixed_one(k, B, nB, p.x, p.m, p.N, aB, w.recB);
            else pack_grad_fp64_one(k, B, nB, p.x, p.m, p.N, aB, (double4_32a *)w.recB);
        }
    t_sync(p);
    const int sp = self ? 1 : 0;
    const double c = c48;  // eps^2 / 48, eps the step of the operator with the 2/3 kick
    const double scale = 2.0 * p.G;
    if (p.csize > 1 || nA <= MT_MAX || p.tcount != SB) {
        mt_grad<MIXED>(p, w.recA, self ? w.recA : w.recB, nA, nB, self, aA, MIXED ? wmax : nullptr, c, at, badbit);
    } else if (MIXED) {
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
    t_sync(p);
    if (t_lead(p)) cnt.grad += self ? (unsigned long long)nA * (nA - 1) : (unsigned long long)nA * nB;
}

// symmetrised time-steps of the set P into tau[n]
template <bool MIXED, int SYM>
__device__ __noinline__ void b_tstep(const SubParams &p, const SubWork &w, const int32_t *P, int n, double *tau, Counts &cnt)
{
    if (n <= 0) return;
    if (n == 1) {
        if (t_id(p) == 0) tau[0] = INFINITY;
        t_sync(p);
        return;
    }
    // exact fly-by derivative: the set's accelerations due to itself first
    const double *acc = nullptr;
    if (SYM & 4) {
        b_acc<MIXED>(p, w, P, n, P, n, true, false, w.aB, nullptr, cnt);
        acc = w.aB;
    }
    for (int k = t_id(p); k < n; k += t_n(p)) {
        if (MIXED) pack_tstep_mixed_one(k, P, n, p.x, p.v, p.m, p.N, p.G, w.recA, acc);
        else pack_tstep_fp64_one(k, P, n, p.x, p.v, p.m, p.N, p.G, (double4_32a *)w.recA, acc);
    }
    t_sync(p);
    if (p.csize > 1 || n <= MT_MAX || p.tcount != SB) {
        mt_tstep<MIXED, SYM>(p, w.recA, n, tau);
    } else if (MIXED) {
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
    t_sync(p);
    if (t_lead(p)) cnt.tstep += (unsigned long long)n * (n - 1);
}

// stable in-place partition of P[0..n) by tau >= pivot; returns |S| (S first, then F).  Every
// block of the team counts |S|; the first block reorders.
__device__ __noinline__ int b_partition(const SubParams &p, int32_t *P, int n, const double *tau, double pivot,
                                        int32_t *tmp)
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
    if (p.crank != 0) {
        t_sync(p);
        return nS;
    }
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
    t_sync(p);
    return nS;
}

__device__ void b_kick(const SubParams &p, const int32_t *L, int n, const double *a, double dt)
{
    for (int k = t_id(p); k < n; k += t_n(p)) {
        const int i = L[k];
        for (int c = 0; c < 3; ++c)
            p.v[c * p.N + i] = __dadd_rn(p.v[c * p.N + i], __dmul_rn(dt, a[c * n + k]));
    }
    t_sync(p);
}

__device__ void b_drift(const SubParams &p, const int32_t *L, int n, double dt)
{
    for (int k = t_id(p); k < n; k += t_n(p)) {
        const int i = L[k];
        for (int c = 0; c < 3; ++c)
            p.x[c * p.N + i] = __dadd_rn(p.x[c * p.N + i], __dmul_rn(dt, p.v[c * p.N + i]));
    }
    t_sync(p);
}

// Algorithm fsi on the set S with the step kc.h (coefficients kc).  cache: 1 keeps the final
// a^SS by particle in p.aC, 2 starts from it (S has not moved between the two fsi(S) of one
// hhs_fsi call, and the deeper levels only touch other particles)
template <bool MIXED>
__device__ __noinline__ void b_fsi(const SubParams &p, const SubWork &w, const int32_t *S, int nS, const StepK &kc,
                                   Counts &cnt, int cache = 0)
{
    const double dt = kc.h;
    if (nS <= 0) return;
    if (t_lead(p)) cnt.fsi += 1;
    if (nS < 2) cache = 0;
    if (cache == 2) {
        if (t_lead(p)) cnt.reused += (unsigned long long)nS * (nS - 1);
        for (int k = t_id(p); k < nS; k += t_n(p)) {
            const int i = S[k];
            for (int c = 0; c < 3; ++c)
                p.v[c * p.N + i] = __dadd_rn(p.v[c * p.N + i], __dmul_rn(kc.k6, p.aC[c * p.N + i]));
        }
        t_sync(p);
    } else {
        b_acc<MIXED>(p, w, S, nS, S, nS, true, false, w.aA, nullptr, cnt);
        b_kick(p, S, nS, w.aA, kc.k6);
    }
    b_drift(p, S, nS, 0.5 * dt);
    b_acc<MIXED>(p, w, S, nS, S, nS, true, true, w.aA, w.wA, cnt);
    b_grad<MIXED>(p, w, S, nS, w.aA, S, nS, w.aA, true, kc.k48, MIXED ? w.wA : nullptr, w.atA, cnt);
    b_kick(p, S, nS, w.atA, kc.k23);
    b_drift(p, S, nS, 0.5 * dt);
    b_acc<MIXED>(p, w, S, nS, S, nS, true, false, w.aA, nullptr, cnt);
    if (cache == 1) {
        for (int k = t_id(p); k < nS; k += t_n(p)) {
            const int i = S[k];
            for (int c = 0; c < 3; ++c) p.aC[c * p.N + i] = w.aA[c * nS + k];
        }
    }
    b_kick(p, S, nS, w.aA, kc.k6);
}

// kick_sf: S kicked by its accelerations due to F, F by those due to S (computed first); with
// the gradient, c48 = tau^2/48 of the level's pivot step tau
template <bool MIXED>
__device__ __noinline__ void b_kick_sf(const SubParams &p, const SubWork &w, const int32_t *S, int nS, const int32_t *F,
                          int nF, double cdt, bool gradient, double c48, Counts &cnt)
{
    if (nS <= 0 || nF <= 0) return;
    b_acc<MIXED>(p, w, S, nS, F, nF, false, gradient, w.aA, gradient ? w.wA : nullptr, cnt);
    b_acc<MIXED>(p, w, F, nF, S, nS, false, gradient, w.aB, gradient ? w.wB : nullptr, cnt);
    if (gradient) {
        b_grad<MIXED>(p, w, S, nS, w.aA, F, nF, w.aB, false, c48, MIXED ? w.wA : nullptr, w.atA, cnt);
        b_grad<MIXED>(p, w, F, nF, w.aB, S, nS, w.aA, false, c48, MIXED ? w.wB : nullptr, w.atB, cnt);
        b_kick(p, S, nS, w.atA, cdt);
        b_kick(p, F, nF, w.atB, cdt);
    } else {
        b_kick(p, S, nS, w.aA, cdt);
        b_kick(p, F, nF, w.aB, cdt);
    }
}

// ---- warp path: the whole subtree of a set of at most 32 particles in one warp ----------
// Lane l holds particle l of the set in registers (FP64 state); sets are lane masks, the
// partition is a ballot and every source is broadcast by shuffle, so a tiny set needs no
// block barrier.  The pair arithmetic is the same as in the block path (pair_bodies.cuh);
// only the summation order differs.
constexpr int WARP_N = 32;

// The lane's particle (FP64 state) and the warp's origin o (the centre of the bounding box of
// the set at entry).  The mixed passes split x - o, not x, into float-float records: x - o is
// at most the set's extent, so a tight pair's separation is resolved to 2^-48 of that extent
// instead of 2^-48 |x| (at the pericentre of a hard binary, r ~ 1e-10 |x|, the absolute
// records would leave a relative error of ~1e-4 in r).  Separations, and so the arithmetic
// of the method, do not depend on the origin.
struct WLane {
    double x[3], v[3], m;
    double o[3];
    double xr[3];  // x - o, drifted with the increments of x (mixed records only)
    // the lane's float-float position record (high part and remainder of x - o) and its FP32
    // mass, renewed whenever the lane drifts: every pass between two drifts reads the same
    // bits, so they are split once (FP64 conversions hold a sub-partition's FP64 unit for
    // about 64 cycles a warp instruction)
    float rh[3], rl[3], mf;
    double ac[3];  // a^SS of the lane's slow set, kept from the first fsi(S) to the second
};

// the lane's float-float record from x - o (mixed passes)
__device__ __forceinline__ void w_record(WLane &L)
{
    for (int c = 0; c < 3; ++c) {
        L.rh[c] = (float)L.xr[c];
        L.rl[c] = (float)(L.xr[c] - (double)L.rh[c]);
    }
    L.mf = (float)L.m;
}

__device__ __forceinline__ float wsh(float v, int j) { return __shfl_sync(0xffffffffu, v, j); }
__device__ __forceinline__ double wshd(double v, int j) { return __shfl_sync(0xffffffffu, v, j); }

// Newtonian pass: every lane sums over the sources j of the uniform mask U with bit j set in
// its own mask mysrc (j != lane).  accurate: the variant that feeds a gradient (Newton-refined
// rsqrt, short folds), also returning max_j m_j / r^3.
template <bool MIXED>
__device__ __noinline__ void w_acc(const SubParams &p, const WLane &L, unsigned U, unsigned mysrc, bool accurate,
                                   double (&a)[3], float &wmax)
{
    const int lane = threadIdx.x & 31;
    const int ipos[1] = {lane};
    float wm[1] = {0.f};
    double res[3] = {0.0, 0.0, 0.0};
    if (MIXED) {
        const float eps2 = (float)p.eps2;
        float H[3] = {0.f, 0.f, 0.f}, Lo[3] = {0.f, 0.f, 0.f};
        float ax[1] = {0.f}, ay[1] = {0.f}, az[1] = {0.f};
        int c = 0;
        AccMixedI<1> I;
        const float hx = L.rh[0], hy = L.rh[1], hz = L.rh[2];
        I.xh[0] = hx; I.yh[0] = hy; I.zh[0] = hz;
        I.xl[0] = L.rl[0];
        I.yl[0] = L.rl[1];
        I.zl[0] = L.rl[2];
        const float mf = L.mf;
        unsigned M = U;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            float4 J0 = make_float4(wsh(hx, j), wsh(hy, j), wsh(hz, j), wsh(mf, j));
            const float4 J1 = make_float4(wsh(I.xl[0], j), wsh(I.yl[0], j), wsh(I.zl[0], j), 0.f);
            if (!((mysrc >> j) & 1u)) J0.w = 0.f;
            if (accurate) acc_mixed_j<1, true, true, true>(J0, J1, I, eps2, j, ipos, ax, ay, az, wm);
            else acc_mixed_j<1, true, false>(J0, J1, I, eps2, j, ipos, ax, ay, az, wm);
            if (++c == 16) {
                fold2(H[0], Lo[0], ax[0]); fold2(H[1], Lo[1], ay[0]); fold2(H[2], Lo[2], az[0]);
                ax[0] = ay[0] = az[0] = 0.f;
                c = 0;
            }
        }
        fold2(H[0], Lo[0], ax[0]); fold2(H[1], Lo[1], ay[0]); fold2(H[2], Lo[2], az[0]);
        for (int q = 0; q < 3; ++q) res[q] = (double)H[q] + (double)Lo[q];
    } else {
        const double4_32a I = make_double4_32a(L.x[0], L.x[1], L.x[2], L.m);
        unsigned M = U;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            double4_32a J = make_double4_32a(wshd(L.x[0], j), wshd(L.x[1], j), wshd(L.x[2], j), wshd(L.m, j));
            if (!((mysrc >> j) & 1u)) J.w = 0.0;
            acc_fp64_j<true>(J, I, p.eps2, j, lane, res[0], res[1], res[2]);
        }
    }
    for (int q = 0; q < 3; ++q) a[q] = g_scale(p.G, res[q]);
    wmax = wm[0];
}

// Gradient pass: lane sums over j in U with bit j of mysrc, using its own acceleration ai
// and the sources' accelerations (each lane's ai); dominant terms (w > thr) in double-float.
template <bool MIXED>
__device__ __noinline__ void w_grad(const SubParams &p, const WLane &L, unsigned U, unsigned mysrc,
                                    const double (&ai)[3], float thr, double (&g)[3])
{
    const int lane = threadIdx.x & 31;
    const int ipos[1] = {lane};
    double res[3] = {0.0, 0.0, 0.0};
    if (MIXED) {
        const float eps2 = (float)p.eps2;
        GradMixedI<1> I;
        split3(L.xr[0], I.xh[0], I.xm[0], I.xl[0]);
        split3(L.xr[1], I.yh[0], I.ym[0], I.yl[0]);
        split3(L.xr[2], I.zh[0], I.zm[0], I.zl[0]);
        I.ahx[0] = trunc12((float)ai[0]);
        I.ahy[0] = trunc12((float)ai[1]);
        I.ahz[0] = trunc12((float)ai[2]);
        I.alx[0] = (float)(ai[0] - (double)I.ahx[0]);
        I.aly[0] = (float)(ai[1] - (double)I.ahy[0]);
        I.alz[0] = (float)(ai[2] - (double)I.ahz[0]);
        const float mf = L.mf;
        const float thrs[1] = {thr};
        BigSlots<1> big;
        init_big(big, lane);
        float H[3] = {0.f, 0.f, 0.f}, Lo[3] = {0.f, 0.f, 0.f};
        float gx[1] = {0.f}, gy[1] = {0.f}, gz[1] = {0.f};
        int c = 0;
        unsigned M = U;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            float4 J0 = make_float4(wsh(I.xh[0], j), wsh(I.yh[0], j), wsh(I.zh[0], j), wsh(mf, j));
            const float4 J1 = make_float4(wsh(I.xm[0], j), wsh(I.ym[0], j), wsh(I.zm[0], j), wsh(I.ahx[0], j));
            const float4 J2 = make_float4(wsh(I.xl[0], j), wsh(I.yl[0], j), wsh(I.zl[0], j), wsh(I.ahy[0], j));
            const float4 J3 = make_float4(wsh(I.ahz[0], j), wsh(I.alx[0], j), wsh(I.aly[0], j), wsh(I.alz[0], j));
            if (!((mysrc >> j) & 1u)) J0.w = 0.f;
            grad_mixed_j<1, true>(J0, J1, J2, J3, I, eps2, j, j, ipos, thrs, big, gx, gy, gz);
            if (++c == 16) {
                fold2(H[0], Lo[0], gx[0]); fold2(H[1], Lo[1], gy[0]); fold2(H[2], Lo[2], gz[0]);
                gx[0] = gy[0] = gz[0] = 0.f;
                c = 0;
            }
        }
        fold2(H[0], Lo[0], gx[0]); fold2(H[1], Lo[1], gy[0]); fold2(H[2], Lo[2], gz[0]);
        // deferred double-float terms: every lane fetches the records of its own slot s (the
        // loop runs to the warp's largest slot count, the shuffles need every lane)
        double bx = 0.0, by = 0.0, bz = 0.0;
        const int nbig = __reduce_max_sync(0xffffffffu, big.n[0]);
#pragma unroll
        for (int s = 0; s < GRAD_SLOTS; ++s) {
            if (s >= nbig) break;
            const int j = big.j[s][0];
            const float4 Q0 = make_float4(wsh(I.xh[0], j), wsh(I.yh[0], j), wsh(I.zh[0], j), wsh(mf, j));
            const float4 Q1 = make_float4(wsh(I.xm[0], j), wsh(I.ym[0], j), wsh(I.zm[0], j), wsh(I.ahx[0], j));
            const float4 Q2 = make_float4(wsh(I.xl[0], j), wsh(I.yl[0], j), wsh(I.zl[0], j), wsh(I.ahy[0], j));
            const float4 Q3 = make_float4(wsh(I.ahz[0], j), wsh(I.alx[0], j), wsh(I.aly[0], j), wsh(I.alz[0], j));
            if (s < big.n[0]) grad_term_df<1>(Q0, Q1, Q2, Q3, I, 0, p.eps2, bx, by, bz);
        }
        res[0] = ((double)H[0] + (double)Lo[0]) + bx;
        res[1] = ((double)H[1] + (double)Lo[1]) + by;
        res[2] = ((double)H[2] + (double)Lo[2]) + bz;
    } else {
        const double4_32a I = make_double4_32a(L.x[0], L.x[1], L.x[2], L.m);
        const double4_32a IA = make_double4_32a(ai[0], ai[1], ai[2], 0.0);
        unsigned M = U;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            double4_32a J = make_double4_32a(wshd(L.x[0], j), wshd(L.x[1], j), wshd(L.x[2], j), wshd(L.m, j));
            const double4_32a JA = make_double4_32a(wshd(ai[0], j), wshd(ai[1], j), wshd(ai[2], j), 0.0);
            if (!((mysrc >> j) & 1u)) J.w = 0.0;
            grad_fp64_j<true>(J, JA, I, IA, p.eps2, j, lane, res[0], res[1], res[2]);
        }
    }
    for (int q = 0; q < 3; ++q) g[q] = 2.0 * p.G * res[q];
}

// symmetrised time-step of the lane's particle over the set P (lane in P)
template <bool MIXED, int SYM>
__device__ __noinline__ double w_tstep(const SubParams &p, const WLane &L, unsigned P, bool &coincident)
{
    const int lane = threadIdx.x & 31;
    const int ipos[1] = {lane};
    coincident = false;
    // exact fly-by derivative: the lanes' accelerations due to the set
    double la[3] = {0.0, 0.0, 0.0};
    if (SYM & 4) {
        float wm;
        w_acc<MIXED>(p, L, P, ((P >> lane) & 1u) ? P : 0u, false, la, wm);
    }
    if (MIXED) {
        TstepMixedI<1> I;
        const float hx = L.rh[0], hy = L.rh[1], hz = L.rh[2];
        I.xh[0] = hx; I.yh[0] = hy; I.zh[0] = hz;
        I.xl[0] = L.rl[0];
        I.yl[0] = L.rl[1];
        I.zl[0] = L.rl[2];
        I.vx[0] = (float)L.v[0]; I.vy[0] = (float)L.v[1]; I.vz[0] = (float)L.v[2];
        I.gm[0] = (p.G == 1.0) ? L.mf : (float)(p.G * L.m);
        I.ax[0] = (float)la[0]; I.ay[0] = (float)la[1]; I.az[0] = (float)la[2];
        const float mf = L.mf;
        const float eta = (float)p.eta, eta15 = 1.5f * eta;
        float best[1] = {INFINITY}, minr2[1] = {INFINITY};
        unsigned M = P;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            const float4 J0 = make_float4(wsh(hx, j), wsh(hy, j), wsh(hz, j), wsh(mf, j));
            const float4 J1 = make_float4(wsh(I.xl[0], j), wsh(I.yl[0], j), wsh(I.zl[0], j), 0.f);
            const float4 JV = make_float4(wsh(I.vx[0], j), wsh(I.vy[0], j), wsh(I.vz[0], j), wsh(I.gm[0], j));
            const float4 JA = (SYM & 4) ? make_float4(wsh(I.ax[0], j), wsh(I.ay[0], j), wsh(I.az[0], j), 0.f)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            tstep_mixed_j<1, SYM, true>(J0, J1, JV, JA, I, eta, eta15, j, ipos, best, minr2);
        }
        coincident = (minr2[0] == 0.f);
        return p.eta * (double)best[0];
    } else {
        const double4_32a I = make_double4_32a(L.x[0], L.x[1], L.x[2], L.m);
        const double4_32a IV = make_double4_32a(L.v[0], L.v[1], L.v[2], p.G * L.m);
        const double4_32a IA = make_double4_32a(la[0], la[1], la[2], 0.0);
        double best = INFINITY, minr2 = INFINITY;
        unsigned M = P;
        while (M) {
            const int j = __ffs(M) - 1;
            M &= M - 1;
            const double4_32a J = make_double4_32a(wshd(I.x, j), wshd(I.y, j), wshd(I.z, j), wshd(I.w, j));
            const double4_32a JV = make_double4_32a(wshd(IV.x, j), wshd(IV.y, j), wshd(IV.z, j), wshd(IV.w, j));
            const double4_32a JA = (SYM & 4) ? make_double4_32a(wshd(IA.x, j), wshd(IA.y, j), wshd(IA.z, j), 0.0)
                                             : make_double4_32a(0.0, 0.0, 0.0, 0.0);
            tstep_fp64_j<SYM, true>(J, JV, JA, I, IV, IA, p.eta, j, lane, best, minr2);
        }
        coincident = (minr2 == 0.0);
        return p.eta * best;
    }
}

__device__ __forceinline__ void w_kick(WLane &L, bool on, const double (&a)[3], double dt)
{
    if (on)
        for (int c = 0; c < 3; ++c) L.v[c] = __dadd_rn(L.v[c], __dmul_rn(dt, a[c]));
}

template <bool MIXED>
__device__ __forceinline__ void w_drift(WLane &L, bool on, double dt)
{
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double d = __dmul_rn(dt, L.v[c]);
            L.x[c] = __dadd_rn(L.x[c], d);
            if (MIXED) L.xr[c] = __dadd_rn(L.xr[c], d);
        }
        if (MIXED) w_record(L);
    }
}

// cache: 1 keeps the final a^SS in the lanes of S (L.ac), 2 starts from it: S has not moved
// between the two fsi(S) of one hhs_fsi call, and the frames in between only touch the lanes
// of F, which are not in S (the same a^SS, bit for bit, as a new pass)
template <bool MIXED>
__device__ void w_fsi(const SubParams &p, WLane &L, unsigned S, const StepK &kc, Counts &cnt, int cache = 0)
{
    const double dt = kc.h;
    if (!S) return;
    const int lane = threadIdx.x & 31;
    const bool in = (S >> lane) & 1u;
    const unsigned src = in ? S : 0u;
    const unsigned long long ns = (unsigned long long)__popc(S);
    if (ns < 2) cache = 0;
    double a[3], at[3], g[3];
    float wm;
    if (cache == 2) {
        for (int q = 0; q < 3; ++q) a[q] = L.ac[q];
    } else {
        w_acc<MIXED>(p, L, S, src, false, a, wm);
    }
    w_kick(L, in, a, kc.k6);
    w_drift<MIXED>(L, in, 0.5 * dt);
    w_acc<MIXED>(p, L, S, src, true, a, wm);
    w_grad<MIXED>(p, L, S, src, a, MIXED ? SLOT_FRACTION * wm : INFINITY, g);
    const double c = kc.k48;
    for (int q = 0; q < 3; ++q) at[q] = a[q] + c * g[q];
    w_kick(L, in, at, kc.k23);
    w_drift<MIXED>(L, in, 0.5 * dt);
    w_acc<MIXED>(p, L, S, src, false, a, wm);
    if (cache == 1 && in)
        for (int q = 0; q < 3; ++q) L.ac[q] = a[q];
    w_kick(L, in, a, kc.k6);
    if (lane == 0) {
        cnt.fsi += 1;
        cnt.acc += (cache == 2 ? 2 : 3) * ns * (ns - 1);
        cnt.grad += ns * (ns - 1);
        if (cache == 2) cnt.reused += ns * (ns - 1);
    }
}

template <bool MIXED>
__device__ void w_kick_sf(const SubParams &p, WLane &L, unsigned S, unsigned F, double cdt, bool gradient,
                          double c48, Counts &cnt)
{
    if (!S || !F) return;
    const int lane = threadIdx.x & 31;
    const bool inS = (S >> lane) & 1u, inF = (F >> lane) & 1u;
    const unsigned src = inS ? F : (inF ? S : 0u);
    const unsigned U = S | F;
    const unsigned long long pairs = 2ull * __popc(S) * __popc(F);
    double a[3];
    float wm;
    w_acc<MIXED>(p, L, U, src, gradient, a, wm);
    if (gradient) {
        double g[3];
        w_grad<MIXED>(p, L, U, src, a, MIXED ? SLOT_FRACTION * wm : INFINITY, g);
        for (int q = 0; q < 3; ++q) a[q] = a[q] + c48 * g[q];
    }
    w_kick(L, inS || inF, a, cdt);
    if (lane == 0) {
        cnt.acc += pairs;
        if (gradient) cnt.grad += pairs;
    }
}

// The subtree of hhs_fsi on the n <= 32 particles Sg[0..n) at depth depth0, run by one warp.
// Returns 0 or an error bit.
template <bool MIXED, int SYM>
__device__ __noinline__ int warp_hhs(const SubParams &p, const int32_t *Sg, int n, double tau0, int depth0,
                                     Counts &cnt)
{
    __shared__ unsigned wf_P[MAXD], wf_S[MAXD];
    __shared__ double wf_tau[MAXD];
    __shared__ int wf_depth[MAXD], wf_pc[MAXD];
    const int lane = threadIdx.x & 31;
    WLane L;
    int gi = 0;
    if (lane < n) {
        gi = Sg[lane];
        for (int c = 0; c < 3; ++c) {
            L.x[c] = p.x[c * p.N + gi];
            L.v[c] = p.v[c * p.N + gi];
        }
        L.m = p.m[gi];
    } else {
        // inactive lanes are never in any set; far, massless placeholders
        for (int c = 0; c < 3; ++c) {
            L.x[c] = 1.0e18 * (c + 1 + lane);
            L.v[c] = 0.0;
        }
        L.m = 0.0;
    }
    // the origin of the mixed records: the centre of the set's bounding box
    for (int c = 0; c < 3; ++c) {
        double lo = (lane < n) ? L.x[c] : INFINITY, hi = (lane < n) ? L.x[c] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        L.o[c] = MIXED ? 0.5 * (lo + hi) : 0.0;
        L.xr[c] = L.x[c] - L.o[c];
        L.ac[c] = 0.0;
    }
    if (MIXED) w_record(L);
    const unsigned all = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
    if (lane == 0) {
        wf_P[0] = all;
        wf_S[0] = 0u;
        wf_tau[0] = tau0;
        wf_depth[0] = depth0;
        wf_pc[0] = 0;
    }
    __syncwarp();
    int sp = 1, err = 0;
    while (sp > 0) {
        const int top = sp - 1;
        const unsigned P = wf_P[top];
        const unsigned S = wf_S[top];
        const double ftau = wf_tau[top];
        const int depth = wf_depth[top], pc = wf_pc[top];
        __syncwarp();
        const unsigned F = P & ~S;
        if (pc == 0) {
            if (depth > p.max_depth) {
                err = ERR_DEPTH;
                break;
            }
            const bool inP = (P >> lane) & 1u;
            bool coin = false;
            const double tau = w_tstep<MIXED, SYM>(p, L, P, coin);
            if (inP && coin) err |= ERR_COINCIDENT;
            if (inP && !(tau > 0.0)) err |= ERR_NONFINITE;
            const unsigned Sn = __ballot_sync(0xffffffffu, inP && tau >= ftau) & P;
            const unsigned Fn = P & ~Sn;
            if (lane == 0) {
                const unsigned long long np = (unsigned long long)__popc(P);
                cnt.hhs += 1;
                cnt.tstep += np * (np - 1);
                cnt.maxdepth = max(cnt.maxdepth, depth);
                const int Lv = min(depth, SUBTREE_STAT_LEVELS - 1);
                atomicAdd(&p.levels[Lv], 1ull);
                atomicAdd(&p.levels[SUBTREE_STAT_LEVELS + Lv], np);
            }
            const StepK &K0 = p.K[depth - p.kdepth0];
            w_kick_sf<MIXED>(p, L, Sn, Fn, K0.k6, false, K0.k48, cnt);
            w_fsi<MIXED>(p, L, Sn, p.K[depth - p.kdepth0 + 1], cnt, 1);
            if (lane == 0) {
                wf_S[top] = Sn;
                wf_pc[top] = 1;
            }
            if (Fn) {
                if (sp >= MAXD) {
                    err |= ERR_DEPTH;
                    break;
                }
                if (lane == 0) {
                    wf_P[sp] = Fn;
                    wf_S[sp] = 0u;
                    wf_tau[sp] = 0.5 * ftau;
                    wf_depth[sp] = depth + 1;
                    wf_pc[sp] = 0;
                }
                sp += 1;
            }
        } else if (pc == 1) {
            const StepK &K0 = p.K[depth - p.kdepth0];
            w_kick_sf<MIXED>(p, L, S, F, K0.k23, true, K0.k48, cnt);
            if (lane == 0) wf_pc[top] = 2;
            if (F) {
                if (lane == 0) {
                    wf_P[sp] = F;
                    wf_S[sp] = 0u;
                    wf_tau[sp] = 0.5 * ftau;
                    wf_depth[sp] = depth + 1;
                    wf_pc[sp] = 0;
                }
                sp += 1;
            }
        } else {
            const StepK &K0 = p.K[depth - p.kdepth0];
            w_fsi<MIXED>(p, L, S, p.K[depth - p.kdepth0 + 1], cnt, 2);
            w_kick_sf<MIXED>(p, L, S, F, K0.k6, false, K0.k48, cnt);
            sp -= 1;
        }
        __syncwarp();
    }
    // a lane's error bits count for the whole warp
    err = __reduce_or_sync(0xffffffffu, err);
    if (lane < n)
        for (int c = 0; c < 3; ++c) {
            p.x[c * p.N + gi] = L.x[c];
            p.v[c * p.N + gi] = L.v[c];
        }
    return err;
}

// Whether a frame of a one-block team runs its fsi(S, tau/2) on warps 1..7 while warp 0 runs
// the whole subtree of hhs_fsi(F, tau/2) (Algorithm hhs-fsi).  The two operators act on the
// disjoint sets S and F (H_S holds only S, H_F only F) and commute; the warp path keeps F in
// registers and touches no workspace, and the sub-team sums in the team's order (mt_map), so
// the result is that of the serial order bit for bit.  sp: the frames on the stack, which the
// serial order would push F onto.
__device__ __forceinline__ bool f_beside(const SubParams &p, int nS, int nF, int sp)
{
    return p.overlap && p.csize == 1 && nS > 0 && nS <= MT_MAX && nF > 0 && nF <= WARP_N && sp < MAXD;
}

// fsi(S, tau/2) (cache as in b_fsi) on warps 1..7 beside warp 0's subtree of F = S + nS (nF
// particles, depth + 1); ends with a block barrier, the warp path's status in *s_e
template <bool MIXED, int SYM>
__device__ __noinline__ void fsi_beside_warp(const SubParams &p, const SubWork &w, const int32_t *S, int nS, int nF,
                                             double ftau, int depth, Counts &cnt, int cache, int *s_e)
{
    if (threadIdx.x < 32) {
        const int e = warp_hhs<MIXED, SYM>(p, S + nS, nF, 0.5 * ftau, depth + 1, cnt);
        if (threadIdx.x == 0) {
            if (e) atomicOr(p.err, e);
            *s_e = e;
        }
    } else {
        SubParams q = p;
        q.tbase = 32;
        q.tcount = SB - 32;
        b_fsi<MIXED>(q, w, S, nS, p.K[depth - p.kdepth0 + 1], cnt, cache);
        if (t_lead(q)) cnt.beside += 1;
    }
    __syncthreads();
}

// One team (a block, or the blocks of one thread-block cluster): n_steps calls of
// hhs_fsi(P, tau0) at depth depth0.  Single-set mode: P, n given, workspace from particle 0.
// Batch mode (offsets != NULL): team t takes cluster c = (cl_index ? cl_index[t] : t), the
// particles [offsets[c], offsets[c+1]) in order, and the workspace region of those particles.
// Every block of a team keeps its own copy of the frame stack and takes the same decisions.
// MINB: blocks per SM the registers must allow.  A single set runs one team, which may use
// up to 255 registers a thread (the mixed kernel takes ~218, without spills); a batch of
// many clusters needs two blocks per SM (128 registers) to run its teams in one wave.
template <bool MIXED, int SYM, int MINB = 1>
__global__ void __launch_bounds__(SB, MINB) k_hhs_subtree(SubParams p0, SubWork w0, const int32_t *__restrict__ P,
                                                    int n_single, const int64_t *__restrict__ offsets,
                                                    const int32_t *__restrict__ cl_index, double tau0,
                                                    int depth0, int n_steps)
{
    __shared__ int f_lo[MAXD], f_n[MAXD], f_ns[MAXD], f_pc[MAXD], f_depth[MAXD];
    __shared__ double f_tau[MAXD];
    __shared__ int s_sp, s_abort, s_we;
    __shared__ StepK s_K[MAXD + 1];
    const int tid = threadIdx.x;
    SubParams p = p0;
    // the step coefficients of every level below depth0: K[r] for tau0 2^-r, the exact
    // power-of-two multiples of tau0's own (read after the first team barrier)
    if (tid <= MAXD) {
        const double sc = __longlong_as_double((long long)(1023 - tid) << 52);  // 2^-tid
        const double k6 = tau0 / 6.0, k23 = 2.0 * tau0 / 3.0, k48 = tau0 * tau0 / 48.0;
        s_K[tid] = StepK{tau0 * sc, k6 * sc, k23 * sc, k48 * (sc * sc)};
    }
    p.K = s_K;
    p.kdepth0 = depth0;
    {
        unsigned r, c;
        asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(c));
        p.crank = (int)r;
        p.csize = (int)c;
    }
    const int team = blockIdx.x / p.csize;
    int off = 0, n = n_single;
    if (offsets) {
        const int c = cl_index ? cl_index[team] : team;
        off = (int)offsets[c];
        n = (int)(offsets[c + 1] - offsets[c]);
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
    w.recA += 6 * (size_t)off;  // 96 bytes per particle
    w.recB += 6 * (size_t)off;
    Counts cnt = {0, 0, 0, 0, 0, depth0, 0, 0};
    if (tid == 0) s_abort = 0;
    for (int step = 0; step < n_steps; ++step) {
        for (int k = t_id(p); k < n; k += t_n(p)) w.perm[k] = offsets ? off + k : P[k];
        if (tid == 0) {
            s_sp = 1;
            f_lo[0] = 0;
            f_n[0] = n;
            f_ns[0] = 0;
            f_pc[0] = 0;
            f_depth[0] = depth0;
            f_tau[0] = tau0;
        }
        t_sync(p);
        while (true) {
            if (s_sp == 0 || s_abort) break;
            const int top = s_sp - 1;
            const int lo = f_lo[top], fn = f_n[top], pc = f_pc[top], depth = f_depth[top];
            const double ftau = f_tau[top];
            int nS = f_ns[top];
            __syncthreads();  // every thread has read the frame before it changes
            int32_t *S = w.perm + lo;
            if (pc == 0 && fn <= WARP_N) {
                // a tiny set: its whole subtree in warp 0 of the team's first block, without
                // block barriers; its status reaches the other blocks through w.xchg
                __shared__ int s_e;
                if (p.crank == 0 && tid < 32) {
                    const int e = warp_hhs<MIXED, SYM>(p, S, fn, ftau, depth, cnt);
                    if (tid == 0) {
                        if (e) atomicOr(p.err, e);
                        s_e = e;
                        if (p.csize > 1) w.xchg[team] = e;
                    }
                }
                t_sync(p);
                if (tid == 0) {
                    const int e = (p.csize > 1) ? *(volatile int *)&w.xchg[team] : s_e;
                    if (e & ERR_DEPTH) s_abort = 1;
                    s_sp -= 1;
                }
            } else if (pc == 0) {
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
                    if (p.crank == 0) {
                        const int L = min(depth, SUBTREE_STAT_LEVELS - 1);
                        atomicAdd(&p.levels[L], 1ull);
                        atomicAdd(&p.levels[SUBTREE_STAT_LEVELS + L], (unsigned long long)fn);
                    }
                }
                b_tstep<MIXED, SYM>(p, w, S, fn, w.tau, cnt);
                nS = b_partition(p, S, fn, w.tau, ftau, w.tmp);
                const int nF = fn - nS;
                const StepK &K0 = p.K[depth - depth0];
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, K0.k6, false, K0.k48, cnt);
                if (f_beside(p, nS, nF, top + 1)) {
                    // fsi(S, tau/2) beside the first hhs_fsi(F, tau/2), which is then done
                    fsi_beside_warp<MIXED, SYM>(p, w, S, nS, nF, ftau, depth, cnt, 1, &s_we);
                    if (tid == 0) {
                        f_ns[top] = nS;
                        f_pc[top] = 1;
                        if (s_we & ERR_DEPTH) s_abort = 1;
                    }
                } else {
                    b_fsi<MIXED>(p, w, S, nS, p.K[depth - depth0 + 1], cnt, 1);
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
                }
            } else if (pc == 1) {
                const int nF = fn - nS;
                const StepK &K0 = p.K[depth - depth0];
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, K0.k23, true, K0.k48, cnt);
                if (f_beside(p, nS, nF, top + 1)) {
                    // the second fsi(S, tau/2) beside the second hhs_fsi(F, tau/2), then the
                    // closing kick_sf: the frame is done
                    fsi_beside_warp<MIXED, SYM>(p, w, S, nS, nF, ftau, depth, cnt, 2, &s_we);
                    const int e = s_we;
                    if (!(e & ERR_DEPTH)) b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, K0.k6, false, K0.k48, cnt);
                    if (tid == 0) {
                        if (e & ERR_DEPTH) s_abort = 1;
                        s_sp -= 1;
                    }
                } else if (tid == 0) {
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
                const StepK &K0 = p.K[depth - depth0];
                b_fsi<MIXED>(p, w, S, nS, p.K[depth - depth0 + 1], cnt, 2);
                b_kick_sf<MIXED>(p, w, S, nS, S + nS, nF, K0.k6, false, K0.k48, cnt);
                if (tid == 0) s_sp -= 1;
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_abort) break;
    }
    // thread 32 leads the sub-team of warps 1..7 and holds the counts of its passes
    if ((tid == 0 || (p.overlap && tid == 32)) && p.crank == 0) {
        atomicAdd(&p.counters[0], cnt.acc);
        atomicAdd(&p.counters[1], cnt.grad);
        atomicAdd(&p.counters[2], cnt.tstep);
        atomicAdd(&p.counters[3], cnt.hhs);
        atomicAdd(&p.counters[4], cnt.fsi);
        atomicMax(&p.counters[5], (unsigned long long)cnt.maxdepth);
        atomicAdd(&p.counters[6], cnt.reused);
        atomicAdd(&p.counters[7], cnt.beside);
    }
}

}  // namespace

cudaError_t launch_subtree(cudaStream_t s, bool mixed, int sym, const SubtreeArgs &a)
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
    p.aC = a.aC;
    p.tbase = 0;
    p.tcount = SB;
    p.overlap = a.overlap ? 1 : 0;
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
    w.xchg = a.xchg;
    const int tb = (a.team_blocks >= 2 && a.team_blocks <= SUBTREE_MAX_CLUSTER) ? a.team_blocks : 1;
    const unsigned nblk = (a.offsets ? (unsigned)a.n_teams : 1u) * (unsigned)tb;
    // teams of several blocks run as thread-block clusters of tb blocks (cluster barriers)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(SB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)tb;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
#define FROST_SUBTREE_CASE(MIX, SYMV)                                                             \
    e = cudaLaunchKernelEx(&cfg, k_hhs_subtree<MIX, SYMV>, p, w, a.P, a.n, a.offsets, a.cl_index, a.tau0, \
                           a.depth0, a.n_steps)
#define FROST_SUBTREE_MIXED_CASE(SYMV)                                                                       \
    e = a.offsets ? cudaLaunchKernelEx(&cfg, k_hhs_subtree<true, SYMV, 2>, p, w, a.P, a.n, a.offsets,        \
                                       a.cl_index, a.tau0, a.depth0, a.n_steps)                              \
                  : cudaLaunchKernelEx(&cfg, k_hhs_subtree<true, SYMV, 1>, p, w, a.P, a.n, a.offsets,        \
                                       a.cl_index, a.tau0, a.depth0, a.n_steps)
    switch ((mixed ? 8 : 0) + sym) {
    case 8 + 0: FROST_SUBTREE_MIXED_CASE(0); break;
    case 8 + 1: FROST_SUBTREE_MIXED_CASE(1); break;
    case 8 + 4: FROST_SUBTREE_MIXED_CASE(4); break;
    case 8 + 5: FROST_SUBTREE_MIXED_CASE(5); break;
    case 8 + 6: FROST_SUBTREE_MIXED_CASE(6); break;
    case 8 + 2: FROST_SUBTREE_MIXED_CASE(2); break;
    case 0: FROST_SUBTREE_CASE(false, 0); break;
    case 1: FROST_SUBTREE_CASE(false, 1); break;
    case 4: FROST_SUBTREE_CASE(false, 4); break;
    case 5: FROST_SUBTREE_CASE(false, 5); break;
    case 6: FROST_SUBTREE_CASE(false, 6); break;
    default: FROST_SUBTREE_CASE(false, 2); break;
    }
#undef FROST_SUBTREE_CASE
#undef FROST_SUBTREE_MIXED_CASE
    return e;
}

}  // namespace frost
