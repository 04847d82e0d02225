// C-ABI of the HHS-FSI hot path (declared in include/frost.h): the context with its device
// particle store, the pair-pass drivers and the HHS-FSI recursion (Algorithm hhs-fsi) with
// FSI steps on the slow sets (Algorithm fsi).
//
// The recursion runs on the host and issues every kernel on the context stream.  Each
// hhs_fsi call synchronises once, after the partition, to learn |S| and |F| (which decide
// the grid shapes and whether to recurse) and to read the device error word; everything
// else is asynchronous.
#include "frost.h"
#include "frost_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <climits>
#include <cstring>
#include <deque>
#include <vector>

using namespace frost;

// message of the last failure in each host thread (frost_last_error); fixed storage, so that
// setting it never allocates
static thread_local char g_last_error[kLastErrorBytes] = {0};

void frost::set_last_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

void frost::clear_last_error() { g_last_error[0] = '\0'; }

namespace {

frost_status fail(frost_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
frost_status fail(frost_status st, const char *fmt, ...)
{
    char buf[kLastErrorBytes];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error("%s", buf);
    return st;
}

#define FROST_CUDA(call)                                                                         \
    do {                                                                                         \
        const cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? FROST_ENOMEM : FROST_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

#define FROST_TRY(expr)                                                                          \
    do {                                                                                         \
        const frost_status s_ = (expr);                                                          \
        if (s_ != FROST_OK) return s_;                                                           \
    } while (0)

// small device/host exchange block
struct Misc {
    int64_t counts[2];  // partition |S|, |F|
    int64_t rel[2];     // list relation: bad/duplicate flag, |A cap B|
    double eres[8];     // energy reduction
    unsigned long long sub[8];  // subtree solver counters (acc, grad, tstep pairs, hhs, fsi, depth,
                                // reused acc pairs, fsi beside the warp path)
    unsigned long long lev[2][SUBTREE_STAT_LEVELS];  // subtree calls / set sizes per depth
    int err;            // sticky device error word
    int pad;
};

struct Timed {
    cudaEvent_t a, b;
    int kind;
    int64_t pairs;
};

}  // namespace

// bytes of packed pair records per particle in recA / recB (up to six 16-byte records: the
// FP64 time-step records with accelerations)
constexpr size_t kRecBytes = 96;

// batch teams: clusters of at least kBatchTeamMinN particles run on kBatchTeamBlocks blocks
constexpr int64_t kBatchTeamMinN = 768;
constexpr int kBatchTeamBlocks = 8;

// sets from this size on take the symmetric time-step pass and wmax prepass (mixed mode,
// frost_opts.sym_cross = 0), and cross pairs of lists from this many pairs on the symmetric
// cross prepass
constexpr int kSymTstepMinN = 8192;
// the smallest j-split, in waves of blocks, of the one-sided pair passes (64k step: 63.9 ms per
// step with the autotuned 1-8 waves, 62.8-62.9 with at least 16 or at least 32)
constexpr int kMinSplitWaves = 16;
constexpr int64_t kSymCrossPrepassMinPairs = int64_t(1) << 26;
// the symmetric force-gradient kick_sf in the default mode: for S x F up to this many pairs,
// where one symmetric launch is faster than the two one-sided directions on two streams (on
// 64k Plummer levels: 0.42 against 0.73 ms at 5212 x 917); at the top levels the symmetric
// kernels execute about as many instructions per interaction as the one-sided ones (their
// B-side reduction and dominant-term ballots cost what the saved pair bodies save)
constexpr int64_t kSymGradMaxPairs = int64_t(1) << 23;

// autotuner rows: the pass kinds, and the Newtonian pass that feeds a gradient (mixed mode:
// its wmax prepass and deferred double-float terms give it a cost profile of its own)
constexpr int TUNE_ACC_ACCURATE = 3;
constexpr int TUNE_ROWS = 4;

// A stream with the scratch that the passes issued on it write (see the pass drivers).
struct Lane {
    cudaStream_t s = nullptr;
    void *recA = nullptr, *recB = nullptr;               // packed records, kRecBytes x N each
    double *part = nullptr;                              // split partials (part_elems)
    double *aA = nullptr, *aB = nullptr, *atA = nullptr, *atB = nullptr;  // [3][N] each
    float *wA = nullptr, *wB = nullptr;                  // max_j m_j / r^3 per particle (mixed)
    unsigned *hist = nullptr;                            // |a| histograms [2][HOT_BINS] (mixed)
    uint32_t *hA = nullptr, *hB = nullptr;               // hot-source masks (mixed)
    double *part_hot = nullptr;                          // hot-source gradient partials
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;    // branch lanes: fork / join events
    bool owns = false;                                   // branch lanes own their buffers
    cudaStream_t shi = nullptr;                          // branch lanes: a stream of the greatest
                                                         // priority for their kick_sf passes
};

struct frost_ctx {
    int N = 0;
    double G = 1.0, eta = 0.2, eps2 = 0.0;
    bool mixed = true;
    int sym = 0;
    int max_depth = 40;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int n_sm = 1;
    double t = 0.0;

    double *x = nullptr, *v = nullptr, *m = nullptr;  // SoA state
    int32_t *all = nullptr;                          // identity list
    int32_t *marks = nullptr;                        // relation marks [N]
    void *recA = nullptr, *recB = nullptr;           // packed records, 64 B x N each
    double *part = nullptr;                          // split partials
    size_t part_elems = 0;
    double *aA = nullptr, *aB = nullptr, *atA = nullptr, *atB = nullptr;  // [3][N] each
    double *aC = nullptr;  // [3][N] by particle: a^SS at the end of the first fsi(S) of hhs_fsi
    double *tau = nullptr;                           // [N]
    float *wA = nullptr, *wB = nullptr;              // max_j m_j / r^3 per particle (mixed)
    unsigned *hist = nullptr;                        // |a| histograms [2][HOT_BINS] (mixed)
    uint32_t *hA = nullptr, *hB = nullptr;           // hot-source masks of aA / aB (mixed)
    double *part_hot = nullptr;                      // FP64 hot-source gradient partials
    size_t part_hot_elems = 0;
    int32_t *perm = nullptr, *ptmp = nullptr;        // subtree solver permutation / scratch
    int subtree_max = 384;                           // sets up to this size run in one block
    int subtree_blocks = 1;                          // blocks (a cluster) per single-set solver launch
    int integrator = FROST_HHS_FSI;                  // frost_integrator of frost_step
    int n_clusters = 0;                              // > 0: batch of independent clusters
    int64_t *d_offsets = nullptr;                    // cluster offsets [n_clusters + 1] (device)
    // batch teams: clusters of at least team_min_n particles run on a thread-block cluster of
    // team_blocks blocks (d_big, largest first), the others on one block each (d_small); the two
    // launches overlap through a side stream
    int32_t *d_big = nullptr, *d_small = nullptr;    // capacity n_clusters each
    int n_big = 0, n_small = 0;
    std::vector<int64_t> h_offsets;                  // cluster offsets (host copy)
    int64_t team_min_n = 768;                        // clusters of at least this size get a team
    int team_blocks = 8;                             // of this many blocks (autotuned)
    int *d_xchg = nullptr;
    cudaStream_t side = nullptr, cap = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the batch step as a CUDA graph (captured once per (dt_pivot, n_steps), then replayed)
    cudaGraphExec_t gexec = nullptr;
    double g_dt = 0.0;
    int64_t g_steps = 0;
    double *d_ecl = nullptr;                         // per-cluster energy sums [n_clusters][8]
    std::vector<double> h_ecl;
    unsigned long long sub_seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long lev_seen[2][SUBTREE_STAT_LEVELS] = {};
    Misc *dmisc = nullptr, *hmisc = nullptr;
    std::vector<int32_t *> lvS, lvF;                 // per-level slow/fast lists
    unsigned *jbest = nullptr;                       // j-side minima of the symmetric time-step pass
    int *pblk = nullptr;                             // per-block slow counts of the partition
    double *pj = nullptr;                            // j-side partials of the symmetric pass
    size_t pj_elems = 0;
    double *part_hot2 = nullptr;                     // B-side hot-source partials of the
                                                     // symmetric gradient pass
    uint8_t *pcnt = nullptr;                         // B-side slot counts of the symmetric
                                                     // gradient kick_sf passes
    int sym_cross = 0;                               // symmetric S x F Newtonian passes in kick_sf:
                                                     // 0 where they fill the GPU, 1 always, -1 never
    Lane main;                                       // the context stream and the buffers above
    std::deque<Lane> branch;                         // per grid level: fsi(S) next to hhs_fsi(F)
                                                     // (a deque: growing it keeps the lanes of
                                                     // the outer levels in place)
    bool branch_streams = true;                      // run the branch lanes concurrently

    frost_stats st{};
    bool timing = false;
    // autotuned wave bound of the j-split per pass kind (0 acc, 1 grad, 2 time-step) and
    // floor(log2 n_active); 0 = the default bound
    int tune_w[TUNE_ROWS][32] = {};
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> event_pool;
    int host_error = 0;  // sticky error already reported
};

namespace {

int ipb(const frost_ctx *c) { return pair_i_per_block(c->mixed); }

int log2_floor(int n)
{
    int b = 0;
    while (b < 30 && (2 << b) <= n) ++b;
    return b;
}

// Launch shape of a pair pass.  waves: the bound on full waves of blocks (0: the autotuned
// or default one); small: 1 for the small-tile kernels, 0 for the 128-record ones, -1 for
// the autotuned choice, else the default: small-tile kernels (mixed mode) when the
// 128-record grid cannot fill one wave.  An autotuned entry is the wave bound, negated for
// the small-tile kernels.
SplitShape shape_for(const frost_ctx *c, int kind, int n_a, int n_s, int waves = 0, int small = -1,
                     int row = -1)
{
    if (row < 0) row = kind;
    const bool chosen = waves <= 0;  // not a candidate the autotuner is timing
    if (waves <= 0 && row >= 0 && row < TUNE_ROWS) {
        const int t = c->tune_w[row][log2_floor(std::max(n_a, 1))];
        if (t != 0) {
            waves = std::abs(t);
            if (small < 0) small = (t < 0) ? 1 : 0;
        }
    }
    if (waves <= 0) waves = 8;
    // Short blocks: the passes of the concurrent branch lanes hold SM slots that the
    // critical path (the recursion and the kick_sf passes, on streams of higher priority)
    // takes as they free; the finer the j-split, the sooner.  The floor does not depend on
    // the branch or timing mode, so every mode runs the same shapes (and gives the same bits).
    if (chosen) waves = std::max(waves, kMinSplitWaves);
    if (!c->mixed) small = 0;
    if (small < 0) {
        const long long nblk = (n_a + ipb(c) - 1) / ipb(c);
        const long long tiles = (n_s + PAIR_TJ - 1) / PAIR_TJ;
        small = (nblk * tiles < (long long)pair_blocks_per_sm(kind, true) * c->n_sm) ? 1 : 0;
    }
    const int tj = small ? PAIR_TJ_SMALL : PAIR_TJ;
    SplitShape sh = small ? choose_shape(n_a, n_s, PAIR_BS_SMALL * PAIR_ILP, pair_blocks_per_sm(kind, true, true),
                                         c->n_sm, waves, tj)
                          : choose_shape(n_a, n_s, ipb(c), pair_blocks_per_sm(kind, c->mixed), c->n_sm, waves);
    sh.small = small;
    // keep the partials inside the scratch buffer
    const long long comps = (kind == PASS_TSTEP) ? 1 : 3;
    while ((long long)sh.nsplit * comps * n_a > (long long)c->part_elems && sh.nsplit > 1) {
        const int tiles = (n_s + tj - 1) / tj;
        const int ns = std::max(1, sh.nsplit / 2);
        const int tps = (tiles + ns - 1) / ns;
        sh.j_per_split = tps * tj;
        sh.nsplit = (n_s + sh.j_per_split - 1) / sh.j_per_split;
    }
    return sh;
}

cudaEvent_t get_event(frost_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

struct TimedScope {
    frost_ctx *c;
    Timed t{};
    bool on;
    cudaStream_t s;
    TimedScope(frost_ctx *c_, cudaStream_t s_, int kind, int64_t pairs) : c(c_), on(c_->timing), s(s_)
    {
        if (!on) return;
        t.a = get_event(c);
        t.b = get_event(c);
        t.kind = kind;
        t.pairs = pairs;
        if (!t.a || !t.b) {
            on = false;
            return;
        }
        cudaEventRecord(t.a, s);
    }
    ~TimedScope()
    {
        if (!on) return;
        cudaEventRecord(t.b, s);
        c->pending.push_back(t);
    }
};

void resolve_timing(frost_ctx *c)
{
    for (const Timed &t : c->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            c->st.timed_launches[t.kind] += 1;
            c->st.timed_ms[t.kind] += ms;
            c->st.timed_pairs[t.kind] += t.pairs;
        }
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->pending.clear();
}

frost_status err_to_status(int e)
{
    if (e & ERR_DEPTH) return fail(FROST_EDEPTH, "hhs_fsi recursion deeper than max_depth");
    if (e & ERR_COINCIDENT)
        return fail(FROST_ECOINCIDENT, "a pair sum is not finite: two distinct particles at zero separation, or "
                                       "a pair term beyond the floating-point range");
    if (e & ERR_NONFINITE) return fail(FROST_ENONFINITE, "non-finite value in a pass (or a non-positive mass / step)");
    if (e & (ERR_INDEX | ERR_DUPLICATE)) return fail(FROST_EINVAL, "index list out of range or repeated");
    if (e & ERR_TIMEOUT) return fail(FROST_ETIMEOUT, "a bounded device wait gave up");
    return FROST_OK;
}

// synchronise the stream, fetch the exchange block and report the device error word
frost_status sync_misc(frost_ctx *c)
{
    FROST_CUDA(cudaMemcpyAsync(c->hmisc, c->dmisc, sizeof(Misc), cudaMemcpyDeviceToHost, c->stream));
    FROST_CUDA(cudaStreamSynchronize(c->stream));
    if (c->timing) resolve_timing(c);
    // fold the subtree solver's device counters into the statistics
    const unsigned long long *sub = c->hmisc->sub;
    for (int k = 0; k < 3; ++k) c->st.subtree_pairs[k] += (int64_t)(sub[k] - c->sub_seen[k]);
    c->st.acc_pairs += (int64_t)(sub[0] - c->sub_seen[0]);
    c->st.grad_pairs += (int64_t)(sub[1] - c->sub_seen[1]);
    c->st.tstep_pairs += (int64_t)(sub[2] - c->sub_seen[2]);
    c->st.hhs_calls += (int64_t)(sub[3] - c->sub_seen[3]);
    c->st.fsi_calls += (int64_t)(sub[4] - c->sub_seen[4]);
    if ((int)sub[5] > c->st.max_depth_seen) c->st.max_depth_seen = (int)sub[5];
    c->st.acc_pairs_reused += (int64_t)(sub[6] - c->sub_seen[6]);
    c->st.subtree_fsi_beside += (int64_t)(sub[7] - c->sub_seen[7]);
    for (int k = 0; k < 8; ++k) c->sub_seen[k] = sub[k];
    for (int q = 0; q < 2; ++q)
        for (int L = 0; L < SUBTREE_STAT_LEVELS; ++L) {
            const unsigned long long cur = c->hmisc->lev[q][L];
            (q == 0 ? c->st.level_calls : c->st.level_particles)[L] += (int64_t)(cur - c->lev_seen[q][L]);
            c->lev_seen[q][L] = cur;
        }
    return err_to_status(c->hmisc->err);
}

// Buffers of a branch lane, the sizes of the main lane's (the context's) buffers.
frost_status alloc_lane_buffers(frost_ctx *c, Lane &L)
{
    const size_t N = (size_t)c->N;
    L.owns = true;
    FROST_CUDA(cudaMalloc(&L.recA, kRecBytes * N));
    FROST_CUDA(cudaMalloc(&L.recB, kRecBytes * N));
    FROST_CUDA(cudaMalloc(&L.part, sizeof(double) * c->part_elems));
    FROST_CUDA(cudaMalloc(&L.aA, sizeof(double) * 3 * N));
    FROST_CUDA(cudaMalloc(&L.aB, sizeof(double) * 3 * N));
    FROST_CUDA(cudaMalloc(&L.atA, sizeof(double) * 3 * N));
    FROST_CUDA(cudaMalloc(&L.atB, sizeof(double) * 3 * N));
    FROST_CUDA(cudaMalloc(&L.wA, sizeof(float) * N));
    FROST_CUDA(cudaMalloc(&L.wB, sizeof(float) * N));
    if (c->mixed) {
        const size_t words = (N + 31) / 32;
        FROST_CUDA(cudaMalloc(&L.hist, sizeof(unsigned) * 2 * HOT_BINS));
        FROST_CUDA(cudaMalloc(&L.hA, sizeof(uint32_t) * words));
        FROST_CUDA(cudaMalloc(&L.hB, sizeof(uint32_t) * words));
        FROST_CUDA(cudaMalloc(&L.part_hot, sizeof(double) * c->part_hot_elems));
    }
    return FROST_OK;
}

void free_lane(Lane &L)
{
    if (L.owns) {
        void *dev[] = {L.recA, L.recB, L.part, L.aA, L.aB, L.atA, L.atB, L.wA, L.wB, L.hist, L.hA, L.hB,
                       L.part_hot};
        for (void *p : dev)
            if (p) cudaFree(p);
    }
    if (L.ev_fork) cudaEventDestroy(L.ev_fork);
    if (L.ev_join) cudaEventDestroy(L.ev_join);
    if (L.owns && L.s) {
        cudaStreamSynchronize(L.s);
        cudaStreamDestroy(L.s);
    }
    if (L.shi) {
        cudaStreamSynchronize(L.shi);
        cudaStreamDestroy(L.shi);
    }
    L = Lane();
}

// ---- pass drivers ------------------------------------------------------------------------
// Every driver issues its work on a Lane: a stream and the scratch that its passes write
// (records, split partials, accelerations, weights, hot masks).  The main lane is the
// context stream with the context's buffers; a branch lane runs the FSI steps of a grid-level
// hhs_fsi call concurrently with the recursion into the fast set (see hhs_fsi).

void pack_pos(frost_ctx *c, Lane &L, const int32_t *list, int n, void *rec)
{
    if (c->mixed) launch_pack_pos_mixed(L.s, list, n, c->x, c->m, c->N, (float4 *)rec);
    else launch_pack_pos_fp64(L.s, list, n, c->x, c->m, c->N, (double4_32a *)rec);
    c->st.kernel_launches += (n > 0);
}

int badbit(const frost_ctx *c) { return c->eps2 == 0.0 ? ERR_COINCIDENT : ERR_NONFINITE; }

// Newtonian accelerations of A from B (self: the same list); writes G * sum into out_soa
// ([3][nA]) and, if given, out_aos ([nA][3]).  With wmax (mixed mode), also the weight
// max_j m_j / r^3 of each particle's dominant term, which the following gradient pass uses.
// With hist (mixed mode, with wmax): the |a| histogram of the pass is added to hist (zeroed by
// the caller) for the hot-source classification of mark_hot.  kick: the kick of A by the
// result, fused into the finalisation.  irec / jrec: records already packed by the caller
// (NULL: packed here into the lane's recA / recB).
bool use_sym_self(const frost_ctx *c, int n) { return c->sym_cross > 0 || (c->sym_cross == 0 && n >= kSymTstepMinN); }

void pass_acc(frost_ctx *c, Lane &L, const int32_t *A, int nA, const int32_t *B, int nB, bool self,
              double *out_soa, double *out_aos, float *wmax = nullptr, unsigned *hist = nullptr,
              KickArgs kick = KickArgs(), const void *irec = nullptr, const void *jrec = nullptr,
              bool wmax_ready = false)
{
    if (nA <= 0) return;
    if (nB <= 0 || (self && nA == 1)) {
        if (out_soa) cudaMemsetAsync(out_soa, 0, sizeof(double) * 3 * nA, L.s);
        if (out_aos) cudaMemsetAsync(out_aos, 0, sizeof(double) * 3 * nA, L.s);
        if (wmax) cudaMemsetAsync(wmax, 0, sizeof(float) * nA, L.s);
        if (hist && c->mixed && out_soa) launch_acc_hist(L.s, out_soa, nA, hist);
        if (kick.v && out_soa) launch_kick(L.s, kick.list, nA, kick.v, kick.N, out_soa, kick.dt);
        return;
    }
    // before a gradient pass (wmax requested) the mixed mode uses the accurate variant on the
    // same position records: a prepass for wmax = max_j m_j / r^3, then the pass with
    // Newton-refined rsqrt, short folds and the terms above wmax / 16 in double-float
    const bool accurate = c->mixed && wmax;
    if (irec) {
        // packed by the caller
    } else {
        pack_pos(c, L, A, nA, L.recA);
        if (!self) pack_pos(c, L, B, nB, L.recB);
    }
    PairArgs a;
    a.irec = irec ? irec : L.recA;
    a.jrec = irec ? jrec : (self ? L.recA : L.recB);
    a.n_a = nA;
    a.n_s = nB;
    a.self_pass = self ? 1 : 0;
    a.eps2 = c->eps2;
    a.part = L.part;
    a.shape = shape_for(c, PASS_ACC, nA, nB, 0, -1, accurate ? TUNE_ACC_ACCURATE : PASS_ACC);
    a.accurate = accurate;
    a.wmax = accurate ? wmax : nullptr;
    a.jlist = B;
    a.m = c->m;
    const int64_t pairs = self ? (int64_t)nA * (nA - 1) : (int64_t)nA * nB;
    {
        TimedScope ts(c, L.s, PASS_ACC, pairs);
        if (accurate && !wmax_ready) {
            // the prepass: each pair once on large sets (the same maxima, bit for bit)
            if (self && use_sym_self(c, nA)) launch_wmax_sym_self(L.s, a.irec, nA, c->eps2, c->n_sm, c->part_elems, wmax);
            else launch_wmax(L.s, a, wmax);
            c->st.kernel_launches += 1;
        }
        launch_acc(L.s, c->mixed, a);
    }
    launch_finalize_vec(L.s, L.part, a.shape.nsplit, nA, c->G, out_soa, out_aos, &c->dmisc->err, badbit(c), kick);
    c->st.kernel_launches += 2;
    c->st.acc_pairs += pairs;
    if (accurate && hist && out_soa) {
        launch_acc_hist(L.s, out_soa, nA, hist);
        c->st.kernel_launches += 1;
    }
}

// Hot sources (mixed mode): after the accurate Newtonian pass of A (nA) against B (nB), marks
// in mask the particles of A with |a| (a_soa) above HOT_KAPPA x the larger median of hist
// (this pass) and hist2 (the companion pass of B against A, n2 values, or NULL); see
// hot_kernels.cu.
void mark_hot(frost_ctx *c, Lane &L, int nA, int nB, bool self, const double *a_soa, const unsigned *hist,
              const unsigned *hist2, int n2, uint32_t *mask)
{
    if (!c->mixed || nA <= 0) return;
    if (nB <= 0 || (self && nA == 1)) {
        cudaMemsetAsync(mask, 0, sizeof(uint32_t) * ((nA + 31) / 32), L.s);
        return;
    }
    launch_hot_mask(L.s, a_soa, nA, hist, hist2, n2, mask);
    c->st.kernel_launches += 1;
}

// the lane's two |a| histograms, zeroed
unsigned *zero_hists(Lane &L)
{
    cudaMemsetAsync(L.hist, 0, sizeof(unsigned) * 2 * HOT_BINS, L.s);
    return L.hist;
}

// gradient of A against B with a_A (soa [3][nA]) and a_B (soa [3][nB]); writes
// a~ = a_A + eps^2/48 g to at_soa / at_aos and g to g_aos (each optional).  wmax: the
// dominant-term weights of A from the Newtonian pass at the same positions (mixed mode).
// kick: the kick of A by a~, fused into the finalisation.  irec / jrec: gradient records
// already packed by the caller (the source records with the hot masses zeroed).
void pass_grad(frost_ctx *c, Lane &L, const int32_t *A, int nA, const double *aA, const int32_t *B, int nB,
               const double *aB, bool self, double eps_grad, double *at_soa, double *at_aos,
               double *g_aos, const float *wmax, const uint32_t *hotB = nullptr,
               KickArgs kick = KickArgs(), const void *irec = nullptr, const void *jrec = nullptr)
{
    if (nA <= 0) return;
    const double cgrad = eps_grad * eps_grad / 48.0;
    if (nB <= 0 || (self && nA == 1)) {
        // no sources: g = 0 and a~ = a
        if (at_soa) cudaMemcpyAsync(at_soa, aA, sizeof(double) * 3 * nA, cudaMemcpyDeviceToDevice, L.s);
        if (at_aos) launch_soa_to_aos(L.s, aA, nA, at_aos);
        if (g_aos) cudaMemsetAsync(g_aos, 0, sizeof(double) * 3 * nA, L.s);
        if (kick.v) launch_kick(L.s, kick.list, nA, kick.v, kick.N, aA, kick.dt);
        return;
    }
    if (!c->mixed) hotB = nullptr;
    if (irec) {
        // packed by the caller
    } else if (c->mixed) {
        // hot sources: masses zeroed in the FP32 source records, their terms summed in
        // double-float by k_grad_hot
        launch_pack_grad_mixed(L.s, A, nA, c->x, c->m, c->N, aA, (float4 *)L.recA, self ? hotB : nullptr);
        if (!self) launch_pack_grad_mixed(L.s, B, nB, c->x, c->m, c->N, aB, (float4 *)L.recB, hotB);
    } else {
        launch_pack_grad_fp64(L.s, A, nA, c->x, c->m, c->N, aA, (double4_32a *)L.recA);
        if (!self) launch_pack_grad_fp64(L.s, B, nB, c->x, c->m, c->N, aB, (double4_32a *)L.recB);
    }
    if (!irec) c->st.kernel_launches += self ? 1 : 2;
    PairArgs a;
    a.irec = irec ? irec : L.recA;
    a.jrec = irec ? jrec : (self ? L.recA : L.recB);
    a.n_a = nA;
    a.n_s = nB;
    a.self_pass = self ? 1 : 0;
    a.eps2 = c->eps2;
    a.part = L.part;
    a.shape = shape_for(c, PASS_GRAD, nA, nB);
    a.wmax = c->mixed ? wmax : nullptr;
    const int64_t pairs = self ? (int64_t)nA * (nA - 1) : (int64_t)nA * nB;
    {
        TimedScope ts(c, L.s, PASS_GRAD, pairs);
        launch_grad(L.s, c->mixed, a);
    }
    int ns_hot = 0;
    if (hotB) {
        ns_hot = hot_grad_splits(nA, nB, c->n_sm);
        while (ns_hot > 1 && (size_t)ns_hot * 3 * nA > c->part_hot_elems) --ns_hot;
        launch_grad_hot(L.s, A, nA, aA, B, nB, aB, hotB, a.self_pass, c->x, c->m, c->N, c->eps2, ns_hot,
                        L.part_hot);
        c->st.kernel_launches += 1;
    }
    launch_finalize_grad(L.s, L.part, a.shape.nsplit, nA, 2.0 * c->G, aA, cgrad, at_soa, at_aos, g_aos,
                         &c->dmisc->err, badbit(c), L.part_hot, ns_hot, kick);
    c->st.kernel_launches += 2;
    c->st.grad_pairs += pairs;
}

// symmetrised time-steps of the set P into tau[nP]
void pass_tstep(frost_ctx *c, Lane &L, const int32_t *P, int nP, double *tau)
{
    if (nP <= 0) return;
    if (nP == 1) {
        // no pair: with zero splits the finalisation writes eta * (+inf)
        launch_finalize_tau(L.s, L.part, 0, 1, c->eta, tau, &c->dmisc->err);
        c->st.kernel_launches += 1;
        return;
    }
    // exact fly-by derivative: the accelerations of the set due to itself, packed with the records
    const double *acc = nullptr;
    if (c->sym & FROST_FLYBY_EXACT) {
        pass_acc(c, L, P, nP, P, nP, true, L.aB, nullptr);
        acc = L.aB;
    }
    if (c->mixed) launch_pack_tstep_mixed(L.s, P, nP, c->x, c->v, c->m, c->N, c->G, (float4 *)L.recA, acc);
    else launch_pack_tstep_fp64(L.s, P, nP, c->x, c->v, c->m, c->N, c->G, (double4_32a *)L.recA, acc);
    const int64_t pairs = (int64_t)nP * (nP - 1);
    // mixed mode, large sets (or always with sym_cross = 1): every pair once for both particles
    if (c->mixed && &L == &c->main && (c->sym_cross > 0 || (c->sym_cross == 0 && nP >= kSymTstepMinN))) {
        const TstepSymShape sh = tstep_sym_shape(nP, c->n_sm, c->part_elems);
        {
            TimedScope ts(c, L.s, PASS_TSTEP, pairs);
            launch_tstep_sym(L.s, L.recA, nP, c->eta, c->sym, sh, L.part, c->jbest, tau, &c->dmisc->err);
        }
        c->st.kernel_launches += 4;
        c->st.tstep_pairs += pairs;
        return;
    }
    PairArgs a;
    a.irec = L.recA;
    a.jrec = L.recA;
    a.n_a = nP;
    a.n_s = nP;
    a.self_pass = 1;
    a.eps2 = 0.0;
    a.part = L.part;
    a.shape = shape_for(c, PASS_TSTEP, nP, nP);
    {
        TimedScope ts(c, L.s, PASS_TSTEP, pairs);
        launch_tstep(L.s, c->mixed, a, c->eta, c->sym, &c->dmisc->err);
    }
    launch_finalize_tau(L.s, L.part, a.shape.nsplit, nP, c->eta, tau, &c->dmisc->err);
    c->st.kernel_launches += 3;
    c->st.tstep_pairs += pairs;
}

// ---- integrator -----------------------------------------------------------------------

void drift(frost_ctx *c, Lane &L, const int32_t *list, int n, double dt)
{
    if (n <= 0) return;
    launch_drift(L.s, list, n, c->x, c->v, c->N, dt);
    c->st.kernel_launches += 1;
}

KickArgs kick_of(frost_ctx *c, const int32_t *list, double dt)
{
    KickArgs k;
    k.list = list;
    k.v = c->v;
    k.N = c->N;
    k.dt = dt;
    return k;
}

// drift of the list, writing the position records of the Newtonian pass that follows into rec
void drift_pack(frost_ctx *c, Lane &L, const int32_t *list, int n, double dt, void *rec)
{
    if (n <= 0) return;
    launch_drift_pack(L.s, list, n, c->x, c->v, c->m, c->N, dt, rec, c->mixed ? 0 : 2);
    c->st.kernel_launches += 1;
}

// position records of the list for a Newtonian pass (both variants read the same records)
void pack_acc(frost_ctx *c, Lane &L, const int32_t *list, int n, void *rec)
{
    if (n <= 0) return;
    pack_pos(c, L, list, n, rec);
}

// gradient records of the list with accelerations a ([3][n]); mixed mode: masses of the hot
// particles (mask) zeroed, their terms are summed in double-float by k_grad_hot
void pack_grad(frost_ctx *c, Lane &L, const int32_t *list, int n, const double *a, void *rec, const uint32_t *mask)
{
    if (n <= 0) return;
    if (c->mixed) launch_pack_grad_mixed(L.s, list, n, c->x, c->m, c->N, a, (float4 *)rec, mask);
    else launch_pack_grad_fp64(L.s, list, n, c->x, c->m, c->N, a, (double4_32a *)rec);
    c->st.kernel_launches += 1;
}

// Algorithm fsi on the set S with step dt.  Each kick is fused into the finalisation of the
// pass that produces its accelerations, and each drift writes the records of the next pass.
// cache: 1 stores the final a^SS by particle in aC; 2 starts from the stored a^SS.  Between
// the two fsi(S) calls of one hhs_fsi only kicks and the deeper levels (other particles)
// run, so S has not moved and the stored values are the ones the pass would recompute.
void fsi(frost_ctx *c, Lane &L, const int32_t *S, int nS, double dt, int cache = 0)
{
    if (nS <= 0) return;
    c->st.fsi_calls += 1;
    if (nS < 2) cache = 0;
    if (cache == 2) {
        launch_kick_by_particle(L.s, S, nS, c->v, c->N, c->aC, dt / 6.0);
        c->st.kernel_launches += 1;
        c->st.acc_pairs_reused += (int64_t)nS * (nS - 1);
    } else {
        pass_acc(c, L, S, nS, S, nS, true, L.aA, nullptr, nullptr, nullptr, kick_of(c, S, dt / 6.0));
    }
    drift_pack(c, L, S, nS, 0.5 * dt, L.recA);
    if (c->mixed) {
        unsigned *h = zero_hists(L);
        pass_acc(c, L, S, nS, S, nS, true, L.aA, nullptr, L.wA, h, KickArgs(), L.recA, L.recA);
        mark_hot(c, L, nS, nS, true, L.aA, h, nullptr, 0, L.hA);
    } else {
        pass_acc(c, L, S, nS, S, nS, true, L.aA, nullptr, L.wA, nullptr, KickArgs(), L.recA, L.recA);
    }
    pass_grad(c, L, S, nS, L.aA, S, nS, L.aA, true, dt, L.atA, nullptr, nullptr, L.wA, L.hA,
              kick_of(c, S, 2.0 * dt / 3.0));
    drift_pack(c, L, S, nS, 0.5 * dt, L.recA);
    KickArgs last = kick_of(c, S, dt / 6.0);
    if (cache == 1) last.store = c->aC;
    pass_acc(c, L, S, nS, S, nS, true, L.aA, nullptr, nullptr, nullptr, last, L.recA, L.recA);
}

// Newtonian accelerations of two disjoint lists due to each other with every pair evaluated
// once (Eq. force-newton-inter, both lines): outA (soa [3][nA]) and outB (soa [3][nB]), each
// list's kick fused into its finalisation.  recA / recB hold the lists' position records.  The
// longer list takes the register side, the shorter one the reduced side (its partials per
// group of i-blocks are then fewer).  Returns false, issuing nothing, when even the finest
// grid of the symmetric kernel (a tile per split) would not fill one wave of the GPU (small
// lists: the two one-sided passes, on two streams, are then faster).
bool pass_acc_sym(frost_ctx *c, Lane &L, const int32_t *A, int nA, const int32_t *B, int nB, double *outA,
                  double *outB, KickArgs kickA, KickArgs kickB, const void *recA, const void *recB, bool force = false)
{
    if (nA <= 0 || nB <= 0) return false;
    const bool swap = nB > nA;
    const int ni = swap ? nB : nA, nj = swap ? nA : nB;
    const SymShape sh = sym_shape(c->mixed ? SYM_ACC_MIXED : SYM_ACC_FP64, ni, nj, c->n_sm, c->part_elems, c->pj_elems);
    if (!force && sh.max_blocks < (long long)sh.blocks_per_wave) return false;
    const int64_t pairs = (int64_t)nA * nB;
    {
        // the kernel delivers both interactions of every pair: its algorithmic work for the
        // roofline is that of two one-sided passes
        TimedScope ts(c, L.s, PASS_ACC, 2 * pairs);
        launch_acc_sym(L.s, c->mixed, swap ? recB : recA, swap ? recA : recB, ni, nj, c->eps2, L.part, c->pj, sh);
    }
    double *out_i = swap ? outB : outA, *out_j = swap ? outA : outB;
    const KickArgs kick_i = swap ? kickB : kickA, kick_j = swap ? kickA : kickB;
    launch_finalize_vec(L.s, L.part, sh.nsplit, ni, c->G, out_i, nullptr, &c->dmisc->err, badbit(c), kick_i);
    launch_finalize_vec(L.s, c->pj, sh.ngroups, nj, -c->G, out_j, nullptr, &c->dmisc->err, badbit(c), kick_j);
    c->st.kernel_launches += 3;
    c->st.acc_pairs += pairs;
    c->st.acc_pairs_symmetric += pairs;
    return true;
}

// The accurate Newtonian sums of two disjoint lists (mixed mode) with every pair once: the
// symmetric wmax prepass and the symmetric pass with the dominant terms of both sides in
// double-float, into M.aA / M.aB (soa), with their |a| histograms in h (A) and h + HOT_BINS
// (B).  M.recA / M.recB hold the lists' position records.  Returns false, issuing nothing,
// unless its finest grid fills one wave of the GPU or force is set.
bool acc_pairwise_defer(frost_ctx *c, Lane &M, const int32_t *A, int nA, const int32_t *B, int nB, unsigned *h,
                        bool force)
{
    if (!c->mixed || nA <= 0 || nB <= 0) return false;
    const bool swap = nB > nA;
    const int ni = swap ? nB : nA, nj = swap ? nA : nB;
    const SymShape sa = sym_shape(SYM_ACC_DEFER, ni, nj, c->n_sm, c->part_elems, c->pj_elems);
    if (!force && sa.max_blocks < (long long)sa.blocks_per_wave) return false;
    const int64_t pairs = (int64_t)nA * nB;
    const int32_t *Li = swap ? B : A, *Lj = swap ? A : B;
    {
        TimedScope ts(c, M.s, PASS_ACC, 0);
        launch_wmax_sym_cross(M.s, M.recA, nA, M.recB, nB, c->eps2, c->n_sm, M.wA, M.wB);
    }
    {
        TimedScope ts(c, M.s, PASS_ACC, 2 * pairs);
        launch_acc_sym_defer(M.s, swap ? M.recB : M.recA, swap ? M.recA : M.recB, ni, nj, c->eps2,
                             swap ? M.wB : M.wA, swap ? M.wA : M.wB, Li, Lj, c->m, M.part, c->pj, c->pcnt, sa);
    }
    launch_finalize_vec(M.s, M.part, sa.nsplit, ni, c->G, swap ? M.aB : M.aA, nullptr, &c->dmisc->err, badbit(c));
    launch_finalize_vec(M.s, c->pj, sa.ngroups, nj, c->G, swap ? M.aA : M.aB, nullptr, &c->dmisc->err, badbit(c));
    launch_acc_hist(M.s, M.aA, nA, h);
    launch_acc_hist(M.s, M.aB, nB, h + HOT_BINS);
    c->st.kernel_launches += 6;
    c->st.acc_pairs += pairs;
    c->st.acc_pairs_symmetric += pairs;
    return true;
}

// The passes of the gradient kick_sf over two disjoint lists A and B with every pair once
// (mixed mode; Eqs. force-newton-inter and force-gradient-inter-1/2, both lines): the
// accurate Newtonian sums of both lists (acc_pairwise_defer), the hot sources of both
// (M.hA / M.hB), the gradient records, and both gradients, finalised per list as
// a~ = a + eps_grad^2/48 g (at_soa, at_aos, g_aos per list, each may be NULL) with the kicks
// kA / kB fused.  M.recA / M.recB hold the lists' position records on entry.  The longer
// list takes the register side.  Returns false, issuing nothing, unless its finest grid
// fills one wave of the GPU or force is set.
bool grad_pairwise_sym(frost_ctx *c, Lane &M, const int32_t *A, int nA, const int32_t *B, int nB, double eps_grad,
                       double *atA_soa, double *atB_soa, double *atA_aos, double *atB_aos, double *gA_aos,
                       double *gB_aos, KickArgs kA, KickArgs kB, bool force)
{
    if (!c->mixed || nA <= 0 || nB <= 0) return false;
    const bool swap = nB > nA;
    const int ni = swap ? nB : nA, nj = swap ? nA : nB;
    const SymShape sg = sym_shape(SYM_GRAD, ni, nj, c->n_sm, c->part_elems, c->pj_elems);
    if (!force && sg.max_blocks < (long long)sg.blocks_per_wave) return false;
    const int64_t pairs = (int64_t)nA * nB;
    unsigned *h = zero_hists(M);
    acc_pairwise_defer(c, M, A, nA, B, nB, h, true);
    mark_hot(c, M, nA, nB, false, M.aA, h, h + HOT_BINS, nB, M.hA);
    mark_hot(c, M, nB, nA, false, M.aB, h + HOT_BINS, h, nA, M.hB);
    pack_grad(c, M, A, nA, M.aA, M.recA, M.hA);
    pack_grad(c, M, B, nB, M.aB, M.recB, M.hB);
    {
        TimedScope ts(c, M.s, PASS_GRAD, 2 * pairs);
        launch_grad_sym(M.s, swap ? M.recB : M.recA, swap ? M.recA : M.recB, ni, nj, c->eps2, swap ? M.wB : M.wA,
                        swap ? M.wA : M.wB, M.part, c->pj, c->pcnt, sg);
    }
    // the double-float terms of the hot sources, per receiving list
    int nsA = hot_grad_splits(nA, nB, c->n_sm), nsB = hot_grad_splits(nB, nA, c->n_sm);
    while (nsA > 1 && (size_t)nsA * 3 * nA > c->part_hot_elems) --nsA;
    while (nsB > 1 && (size_t)nsB * 3 * nB > c->part_hot_elems) --nsB;
    launch_grad_hot(M.s, A, nA, M.aA, B, nB, M.aB, M.hB, 0, c->x, c->m, c->N, c->eps2, nsA, c->part_hot);
    launch_grad_hot(M.s, B, nB, M.aB, A, nA, M.aA, M.hA, 0, c->x, c->m, c->N, c->eps2, nsB, c->part_hot2);
    const double cgrad = eps_grad * eps_grad / 48.0;
    const double *ph_i = swap ? c->part_hot2 : c->part_hot, *ph_j = swap ? c->part_hot : c->part_hot2;
    const int ns_i = swap ? nsB : nsA, ns_j = swap ? nsA : nsB;
    launch_finalize_grad(M.s, M.part, sg.nsplit, ni, 2.0 * c->G, swap ? M.aB : M.aA, cgrad, swap ? atB_soa : atA_soa,
                         swap ? atB_aos : atA_aos, swap ? gB_aos : gA_aos, &c->dmisc->err, badbit(c), ph_i, ns_i,
                         swap ? kB : kA);
    launch_finalize_grad(M.s, c->pj, sg.ngroups, nj, 2.0 * c->G, swap ? M.aA : M.aB, cgrad, swap ? atA_soa : atB_soa,
                         swap ? atA_aos : atB_aos, swap ? gA_aos : gB_aos, &c->dmisc->err, badbit(c), ph_j, ns_j,
                         swap ? kA : kB);
    c->st.kernel_launches += 5;
    c->st.grad_pairs += pairs;
    c->st.grad_pairs_symmetric += pairs;
    return true;
}

// Runs on `exec` what a branch lane issues: the branch lane itself when the branches run
// concurrently, else its buffers on the context stream (timing mode, or concurrency off).
// critical: work on the step's critical path (the F side of a kick_sf) takes the lane's
// stream of the greatest priority; the lane's fsi(S) steps take its stream of the lowest, so
// that they yield to the recursion and to the kick_sf passes of the levels below.
struct Branch {
    frost_ctx *c;
    Lane *B;
    Lane exec;
    bool concurrent;
    bool open = false;
    Branch(frost_ctx *c_, Lane *B_, bool critical = false) : c(c_), B(B_), exec(*B_)
    {
        concurrent = c->branch_streams && !c->timing;
        if (!concurrent) exec.s = c->stream;
        else if (critical && B_->shi) exec.s = B_->shi;
    }
    // the branch continues after everything issued so far on the context stream
    void fork()
    {
        if (!concurrent) return;
        cudaEventRecord(B->ev_fork, c->stream);
        cudaStreamWaitEvent(exec.s, B->ev_fork, 0);
        open = true;
    }
    // the context stream continues after everything issued on the branch
    void join()
    {
        if (!open) return;
        cudaEventRecord(B->ev_join, exec.s);
        cudaStreamWaitEvent(c->stream, B->ev_join, 0);
        open = false;
    }
    ~Branch() { join(); }
};

// kick_sf: S kicked by its accelerations due to F, F by those due to S, both computed before
// either kick.  Accelerations depend on positions only, so each list's kick is fused into its
// own pass; both lists are packed once (S in recA, F in recB of the main lane) for the two
// directions.  The two directions are independent: with a branch lane Bl (idle between the
// fsi(S) steps of its level) the F-side passes run on it, concurrently with the S-side passes
// on the main lane, writing their partials in the branch's scratch and their results in the
// main lane's buffers.
void kick_sf(frost_ctx *c, Lane &M, Lane *Bl, const int32_t *S, int nS, const int32_t *F, int nF, double cdt,
             bool gradient, double tau_pivot)
{
    if (nS <= 0 || nF <= 0) return;
    pack_acc(c, M, S, nS, M.recA);
    pack_acc(c, M, F, nF, M.recB);
    Branch br(c, Bl ? Bl : &M, true);
    if (!Bl) br.concurrent = false;
    Lane &X = Bl ? br.exec : M;
    if (!gradient) {
        // each S x F pair once, when the symmetric grid fills the GPU
        if (c->sym_cross >= 0 && pass_acc_sym(c, M, S, nS, F, nF, M.aA, M.aB, kick_of(c, S, cdt),
                                              kick_of(c, F, cdt), M.recA, M.recB, c->sym_cross > 0))
            return;
        br.fork();
        pass_acc(c, M, S, nS, F, nF, false, M.aA, nullptr, nullptr, nullptr, kick_of(c, S, cdt), M.recA, M.recB);
        pass_acc(c, X, F, nF, S, nS, false, M.aB, nullptr, nullptr, nullptr, kick_of(c, F, cdt), M.recB, M.recA);
        return;  // joined by br
    }
    // each S x F pair once for both sides: always with sym_cross = 1, else for small lists
    if (c->sym_cross >= 0 && (c->sym_cross > 0 || (int64_t)nS * nF <= kSymGradMaxPairs) &&
        grad_pairwise_sym(c, M, S, nS, F, nF, tau_pivot, M.atA, M.atB, nullptr, nullptr, nullptr, nullptr,
                          kick_of(c, S, cdt), kick_of(c, F, cdt), true))
        return;
    unsigned *h = c->mixed ? zero_hists(M) : nullptr;
    // the prepasses of both accurate passes in one symmetric kernel (each pair once), where
    // the lists are large
    bool wready = false;
    if (c->mixed && c->sym_cross >= 0 && (c->sym_cross > 0 || (int64_t)nS * nF >= kSymCrossPrepassMinPairs)) {
        TimedScope ts(c, M.s, PASS_ACC, 0);
        launch_wmax_sym_cross(M.s, M.recA, nS, M.recB, nF, c->eps2, c->n_sm, M.wA, M.wB);
        c->st.kernel_launches += 1;
        wready = true;
    }
    br.fork();
    pass_acc(c, M, S, nS, F, nF, false, M.aA, nullptr, M.wA, h, KickArgs(), M.recA, M.recB, wready);
    pass_acc(c, X, F, nF, S, nS, false, M.aB, nullptr, M.wB, h ? h + HOT_BINS : nullptr, KickArgs(), M.recB,
             M.recA, wready);
    br.join();
    if (h) {
        mark_hot(c, M, nS, nF, false, M.aA, h, h + HOT_BINS, nF, M.hA);
        mark_hot(c, M, nF, nS, false, M.aB, h + HOT_BINS, h, nS, M.hB);
    }
    pack_grad(c, M, S, nS, M.aA, M.recA, c->mixed ? M.hA : nullptr);
    pack_grad(c, M, F, nF, M.aB, M.recB, c->mixed ? M.hB : nullptr);
    br.fork();
    pass_grad(c, M, S, nS, M.aA, F, nF, M.aB, false, tau_pivot, M.atA, nullptr, nullptr, M.wA, M.hB,
              kick_of(c, S, cdt), M.recA, M.recB);
    pass_grad(c, X, F, nF, M.aB, S, nS, M.aA, false, tau_pivot, M.atB, nullptr, nullptr, M.wB, M.hA,
              kick_of(c, F, cdt), M.recB, M.recA);
}

frost_status ensure_level(frost_ctx *c, int depth)
{
    while ((int)c->lvS.size() <= depth) {
        int32_t *S = nullptr, *F = nullptr;
        FROST_CUDA(cudaMalloc(&S, sizeof(int32_t) * c->N));
        if (cudaMalloc(&F, sizeof(int32_t) * c->N) != cudaSuccess) {
            cudaFree(S);
            return fail(FROST_ENOMEM, "level list allocation failed");
        }
        c->lvS.push_back(S);
        c->lvF.push_back(F);
    }
    return FROST_OK;
}

// the whole subtree of hhs_fsi(P, tau) in one thread block (single launch, no sync), on the
// main lane
void hhs_subtree(frost_ctx *c, const int32_t *P, int nP, double tau, int depth)
{
    SubtreeArgs a;
    a.x = c->x;
    a.v = c->v;
    a.m = c->m;
    a.N = c->N;
    a.G = c->G;
    a.eta = c->eta;
    a.eps2 = c->eps2;
    a.max_depth = c->max_depth;
    a.err = &c->dmisc->err;
    a.counters = c->dmisc->sub;
    a.levels = &c->dmisc->lev[0][0];
    a.aC = c->aC;
    a.perm = c->perm;
    a.tmp = c->ptmp;
    a.tau = c->tau;
    a.aA = c->aA;
    a.aB = c->aB;
    a.atA = c->atA;
    a.atB = c->atB;
    a.wA = c->wA;
    a.wB = c->wB;
    a.recA = c->recA;
    a.recB = c->recB;
    a.P = P;
    a.n = nP;
    a.tau0 = tau;
    a.depth0 = depth;
    a.n_steps = 1;
    a.team_blocks = c->subtree_blocks;
    a.xchg = c->d_xchg;
    a.overlap = c->branch_streams;
    {
        TimedScope ts(c, c->stream, PASS_SUBTREE, 0);
        // a launch error is also left for the cudaGetLastError() of the calling entry point
        (void)launch_subtree(c->stream, c->mixed, c->sym, a);
    }
    c->st.kernel_launches += 1;
    c->st.subtree_launches += 1;
}

// The branch lane of grid level `depth`: its own scratch (the size of the main lane's) and a
// non-blocking stream of the lowest priority, so that the recursion on the context stream,
// the critical path of the step, is scheduled first.  Allocated on first use.
frost_status branch_lane(frost_ctx *c, int depth, Lane **out)
{
    while ((int)c->branch.size() <= depth) c->branch.push_back(Lane());
    Lane &B = c->branch[depth];
    if (!B.s) {
        int lo = 0, hi = 0;
        FROST_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        // fsi(S) of level d must end before that level's next kick_sf, which comes after the whole
        // recursion below it: the outer the level, the more slack, so the lower the priority
        // (lowest at the top level, one step up per level, always below the greatest, which the
        // kick_sf passes of every level take)
        const int prio = (lo > hi) ? lo - std::min(depth, lo - hi - 1) : lo;
        FROST_CUDA(cudaStreamCreateWithPriority(&B.s, cudaStreamNonBlocking, prio));
        FROST_CUDA(cudaStreamCreateWithPriority(&B.shi, cudaStreamNonBlocking, hi));
        FROST_CUDA(cudaEventCreateWithFlags(&B.ev_fork, cudaEventDisableTiming));
        FROST_CUDA(cudaEventCreateWithFlags(&B.ev_join, cudaEventDisableTiming));
        FROST_TRY(alloc_lane_buffers(c, B));
    }
    *out = &B;
    return FROST_OK;
}

// The first part of hhs_fsi(P, tau): nothing for an empty set, the single-block subtree
// launch for a small set, else the time-step pass and the partition of a grid level, issued
// on the context stream without waiting for them.  done: nothing is left for hhs_tail.
struct HhsHead {
    bool done = true;
    const int32_t *P = nullptr;
    int nP = 0;
    double tau = 0.0;
    int depth = 0;
};

frost_status hhs_head(frost_ctx *c, const int32_t *P, int nP, double tau, int depth, HhsHead &h)
{
    h = HhsHead();
    h.P = P;
    h.nP = nP;
    h.tau = tau;
    h.depth = depth;
    if (nP <= 0) return FROST_OK;
    if (depth > c->max_depth)
        return fail(FROST_EDEPTH, "hhs_fsi deeper than max_depth=%d (|P|=%d, tau_pivot=%g)",
                    c->max_depth, nP, tau);
    if (nP <= c->subtree_max && c->max_depth < SUBTREE_MAX_FRAMES) {
        hhs_subtree(c, P, nP, tau, depth);
        return FROST_OK;
    }
    c->st.hhs_calls += 1;
    if (depth > c->st.max_depth_seen) c->st.max_depth_seen = depth;
    {
        const int Lv = std::min(depth, FROST_STATS_LEVELS - 1);
        c->st.level_calls[Lv] += 1;
        c->st.level_particles[Lv] += nP;
    }
    FROST_TRY(ensure_level(c, depth));
    Lane &M = c->main;
    pass_tstep(c, M, P, nP, c->tau);
    launch_partition(M.s, P, nP, c->tau, tau, c->lvS[depth], c->lvF[depth], c->dmisc->counts, c->pblk);
    c->st.kernel_launches += nP >= PART_MULTI_MIN ? 2 : 1;
    h.done = false;
    return FROST_OK;
}

frost_status hhs_tail(frost_ctx *c, const HhsHead &h);

// Algorithm hhs-fsi on the set P (device list, nP entries) with pivot step tau.
frost_status hhs_fsi(frost_ctx *c, const int32_t *P, int nP, double tau, int depth)
{
    HhsHead h;
    FROST_TRY(hhs_head(c, P, nP, tau, depth, h));
    return hhs_tail(c, h);
}

// The rest of hhs_fsi(P) after hhs_head: read |S| and |F|, then the kicks, the two fsi(S)
// steps and the two recursions into F.  The operators of fsi(S, tau/2) and hhs_fsi(F, tau/2)
// act on disjoint particles (H_S holds only S, H_F only F), so each fsi(S) runs on the level's
// branch lane concurrently with the recursion into F on the context stream; the kick_sf
// between them joins both.  The head of the recursion (its time-step pass and partition, or
// its subtree launch) is issued before the branch's fsi(S), so that the context stream, the
// critical path, has work while the host issues the branch.  The arithmetic, and so every
// result, is that of the serial order.
frost_status hhs_tail(frost_ctx *c, const HhsHead &h)
{
    if (h.done) return FROST_OK;
    const double tau = h.tau;
    const int depth = h.depth;
    Lane &M = c->main;
    int32_t *S = c->lvS[depth], *F = c->lvF[depth];
    FROST_TRY(sync_misc(c));
    const int nS = (int)c->hmisc->counts[0];
    const int nF = (int)c->hmisc->counts[1];
    if (nF == 0 || nS == 0) {
        // one of the two sets is empty: no kick_sf, and the two half steps of the other set
        // follow each other on the context stream
        fsi(c, M, S, nS, 0.5 * tau, 1);
        FROST_TRY(hhs_fsi(c, F, nF, 0.5 * tau, depth + 1));
        FROST_TRY(hhs_fsi(c, F, nF, 0.5 * tau, depth + 1));
        fsi(c, M, S, nS, 0.5 * tau, 2);
        return FROST_OK;
    }
    Lane *Bl = nullptr;
    FROST_TRY(branch_lane(c, depth, &Bl));
    kick_sf(c, M, Bl, S, nS, F, nF, tau / 6.0, false, tau);
    {
        Branch br(c, Bl);
        br.fork();
        HhsHead child;
        FROST_TRY(hhs_head(c, F, nF, 0.5 * tau, depth + 1, child));
        fsi(c, br.exec, S, nS, 0.5 * tau, 1);
        FROST_TRY(hhs_tail(c, child));
    }
    kick_sf(c, M, Bl, S, nS, F, nF, 2.0 * tau / 3.0, true, tau);
    {
        Branch br(c, Bl);
        br.fork();
        HhsHead child;
        FROST_TRY(hhs_head(c, F, nF, 0.5 * tau, depth + 1, child));
        fsi(c, br.exec, S, nS, 0.5 * tau, 2);
        FROST_TRY(hhs_tail(c, child));
    }
    kick_sf(c, M, Bl, S, nS, F, nF, tau / 6.0, false, tau);
    return FROST_OK;
}

// validate a caller list (range and repeats); NULL lists are valid by construction
frost_status check_list(frost_ctx *c, const int32_t *L, int n)
{
    if (!L || n <= 0) return FROST_OK;
    launch_list_relation(c->stream, nullptr, 0, L, n, c->N, c->marks, c->dmisc->rel);
    FROST_TRY(sync_misc(c));
    if (c->hmisc->rel[0]) return fail(FROST_EINVAL, "index list has an out-of-range or repeated index");
    return FROST_OK;
}

frost_status check_sizes(frost_ctx *c, int64_t n, const char *what)
{
    if (n < 0 || n > c->N) return fail(FROST_EINVAL, "%s = %lld outside [0, %d]", what, (long long)n, c->N);
    return FROST_OK;
}

// The team split of a batch context: clusters of at least min_n particles run on a
// thread-block cluster of `blocks` blocks (largest first), the others on one block each (largest
// first, so that the block scheduler starts them first).  Drops the captured step graph.
frost_status set_teams(frost_ctx *c, int64_t min_n, int blocks)
{
    const int nc = c->n_clusters;
    const int64_t *off = c->h_offsets.data();
    std::vector<int32_t> order(nc);
    for (int k = 0; k < nc; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    std::vector<int32_t> big, small;
    for (int32_t k : order) (off[k + 1] - off[k] >= min_n ? big : small).push_back(k);
    c->n_big = (int)big.size();
    c->n_small = (int)small.size();
    if (c->n_big)
        FROST_CUDA(cudaMemcpy(c->d_big, big.data(), sizeof(int32_t) * c->n_big, cudaMemcpyHostToDevice));
    if (c->n_small)
        FROST_CUDA(cudaMemcpy(c->d_small, small.data(), sizeof(int32_t) * c->n_small, cudaMemcpyHostToDevice));
    c->team_min_n = min_n;
    c->team_blocks = blocks;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return FROST_OK;
}

void destroy(frost_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (Lane &L : c->branch) free_lane(L);
    for (const Timed &t : c->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    for (auto p : c->lvS) cudaFree(p);
    for (auto p : c->lvF) cudaFree(p);
    if (c->d_offsets) cudaFree(c->d_offsets);
    if (c->d_big) cudaFree(c->d_big);
    if (c->d_small) cudaFree(c->d_small);
    if (c->d_xchg) cudaFree(c->d_xchg);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->d_ecl) cudaFree(c->d_ecl);
    void *dev[] = {c->x, c->v, c->m, c->all, c->marks, c->recA, c->recB, c->part,
                   c->aA, c->aB, c->atA, c->atB, c->aC, c->tau, c->wA, c->wB, c->perm,
                   c->ptmp, c->dmisc, c->hist, c->hA, c->hB, c->part_hot, c->part_hot2, c->pcnt, c->pj, c->jbest, c->pblk};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (c->hmisc) cudaFreeHost(c->hmisc);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // namespace

// ============================================================================================
// C-ABI
// ============================================================================================
extern "C" {

void frost_default_opts(frost_opts *opt)
{
    if (!opt) return;
    opt->precision = FROST_PREC_MIXED;
    opt->sym = FROST_SYM_HARMONIC;
    opt->eps_soft = 0.0;
    opt->max_depth = 40;
    opt->cuda_stream = nullptr;
    opt->subtree_max = 0;
    opt->subtree_blocks = 0;
    opt->integrator = FROST_HHS_FSI;
    opt->branch_streams = 0;
    opt->sym_cross = 0;
}

const char *frost_last_error(void) { return g_last_error; }

const char *frost_version(void) { return "frost-gb300 0.3 (sm_103a)"; }

static frost_status init_impl(frost_ctx **out, int64_t n, const double *m, const double *x,
                              const double *v, double G, double eta, const frost_opts *opt,
                              int32_t n_clusters, const int64_t *offsets);

frost_status frost_init(frost_ctx **out, int64_t n, const double *m, const double *x, const double *v,
                        double G, double eta, const frost_opts *opt)
{
    return init_impl(out, n, m, x, v, G, eta, opt, 0, nullptr);
}

frost_status frost_init_batch(frost_ctx **out, int32_t n_clusters, const int64_t *offsets,
                              const double *m, const double *x, const double *v, double G, double eta,
                              const frost_opts *opt)
{
    clear_last_error();
    if (!out) return fail(FROST_EINVAL, "ctx pointer is NULL");
    *out = nullptr;
    if (n_clusters < 1 || !offsets) return fail(FROST_EINVAL, "need n_clusters >= 1 and offsets");
    if (offsets[0] != 0) return fail(FROST_EINVAL, "offsets[0] must be 0");
    for (int k = 0; k < n_clusters; ++k)
        if (offsets[k + 1] <= offsets[k]) return fail(FROST_EINVAL, "offsets must increase (cluster %d empty)", k);
    return init_impl(out, offsets[n_clusters], m, x, v, G, eta, opt, n_clusters, offsets);
}

static frost_status init_impl(frost_ctx **out, int64_t n, const double *m, const double *x,
                              const double *v, double G, double eta, const frost_opts *opt,
                              int32_t n_clusters, const int64_t *offsets)
{
    clear_last_error();
    if (!out) return fail(FROST_EINVAL, "ctx pointer is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(FROST_EINVAL, "n = %lld out of range", (long long)n);
    if (!m || !x || !v) return fail(FROST_EINVAL, "m, x and v are required");
    if (!(G > 0.0) || !std::isfinite(G) || !(eta > 0.0) || !std::isfinite(eta))
        return fail(FROST_EINVAL, "G and eta must be finite and positive");
    frost_opts o;
    frost_default_opts(&o);
    if (opt) o = *opt;
    if (o.precision != FROST_PREC_FP64 && o.precision != FROST_PREC_MIXED)
        return fail(FROST_EINVAL, "unknown precision %d", o.precision);
    if (o.sym < 0 || (o.sym & ~FROST_FLYBY_EXACT) > 2 || o.sym > 6)
        return fail(FROST_EINVAL, "unknown symmetrisation %d", o.sym);
    if (!(o.eps_soft >= 0.0) || !std::isfinite(o.eps_soft)) return fail(FROST_EINVAL, "bad softening");
    if (o.integrator != FROST_HHS_FSI && o.integrator != FROST_HOLD2)
        return fail(FROST_EINVAL, "unknown integrator %d", o.integrator);
    if (o.integrator == FROST_HOLD2 && n_clusters > 0)
        return fail(FROST_EINVAL, "the HOLD integrator runs on single-set contexts only");

    if (o.subtree_blocks < 0 || o.subtree_blocks > SUBTREE_MAX_CLUSTER)
        return fail(FROST_EINVAL, "subtree_blocks must be 0..%d", SUBTREE_MAX_CLUSTER);

    frost_ctx *c = new (std::nothrow) frost_ctx();
    if (!c) return fail(FROST_ENOMEM, "host allocation failed");
    c->N = (int)n;
    c->G = G;
    c->eta = eta;
    c->eps2 = o.eps_soft * o.eps_soft;
    c->mixed = (o.precision == FROST_PREC_MIXED);
    c->sym = o.sym;
    c->max_depth = o.max_depth > 0 ? o.max_depth : 40;
    c->subtree_max = o.subtree_max == 0 ? 384 : (o.subtree_max < 0 ? 0 : o.subtree_max);
    c->subtree_blocks = o.subtree_blocks == 0 ? 1 : o.subtree_blocks;
    c->integrator = o.integrator;

    auto bail = [&](frost_status st) {
        destroy(c);
        return st;
    };
#define INIT_CUDA(call)                                                                          \
    do {                                                                                         \
        const cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                                   \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? FROST_ENOMEM : FROST_ECUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                           \
    } while (0)

    INIT_CUDA(cudaGetDevice(&c->device));
    INIT_CUDA(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
    // NULL selects the legacy default stream, which is ordered with every blocking stream
    c->stream = (cudaStream_t)o.cuda_stream;
    const size_t N = (size_t)n;
    INIT_CUDA(cudaMalloc(&c->x, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->v, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->m, sizeof(double) * N));
    INIT_CUDA(cudaMalloc(&c->all, sizeof(int32_t) * N));
    INIT_CUDA(cudaMalloc(&c->marks, sizeof(int32_t) * N));
    INIT_CUDA(cudaMalloc(&c->recA, kRecBytes * N));
    INIT_CUDA(cudaMalloc(&c->recB, kRecBytes * N));
    int bps = 1;
    for (int k = 0; k < 3; ++k) bps = std::max(bps, pair_blocks_per_sm(k, c->mixed));
    bps = std::max(bps, pair_blocks_per_sm(PASS_ACC, false));
    c->part_elems = 3 * std::max(N, (size_t)8 * c->n_sm * bps * PAIR_BS * PAIR_ILP);
    INIT_CUDA(cudaMalloc(&c->part, sizeof(double) * c->part_elems));
    INIT_CUDA(cudaMalloc(&c->aA, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->aB, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->atA, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->atB, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->aC, sizeof(double) * 3 * N));
    INIT_CUDA(cudaMalloc(&c->tau, sizeof(double) * N));
    INIT_CUDA(cudaMalloc(&c->wA, sizeof(float) * N));
    INIT_CUDA(cudaMalloc(&c->wB, sizeof(float) * N));
    if (c->mixed) {
        const size_t words = (N + 31) / 32;
        c->part_hot_elems = 3 * std::max(N, (size_t)HOT_MAX_SPLITS * c->n_sm * 256);
        INIT_CUDA(cudaMalloc(&c->hist, sizeof(unsigned) * 2 * HOT_BINS));
        INIT_CUDA(cudaMalloc(&c->hA, sizeof(uint32_t) * words));
        INIT_CUDA(cudaMalloc(&c->hB, sizeof(uint32_t) * words));
        INIT_CUDA(cudaMalloc(&c->part_hot, sizeof(double) * c->part_hot_elems));
        INIT_CUDA(cudaMalloc(&c->part_hot2, sizeof(double) * c->part_hot_elems));
    }
    c->pj_elems = 3 * 8 * N;
    INIT_CUDA(cudaMalloc(&c->pj, sizeof(double) * c->pj_elems));
    if (c->mixed) INIT_CUDA(cudaMalloc(&c->pcnt, (c->pj_elems / 3) * SYM_PCNT_WARPS));
    INIT_CUDA(cudaMalloc(&c->jbest, sizeof(unsigned) * N));
    INIT_CUDA(cudaMalloc(&c->pblk, sizeof(int) * (size_t)partition_blocks((int)N)));
    INIT_CUDA(cudaMalloc(&c->perm, sizeof(int32_t) * N));
    INIT_CUDA(cudaMalloc(&c->ptmp, sizeof(int32_t) * N));
    if (n_clusters > 0) {
        c->n_clusters = n_clusters;
        INIT_CUDA(cudaMalloc(&c->d_offsets, sizeof(int64_t) * (n_clusters + 1)));
        INIT_CUDA(cudaMemcpy(c->d_offsets, offsets, sizeof(int64_t) * (n_clusters + 1), cudaMemcpyHostToDevice));
        INIT_CUDA(cudaMalloc(&c->d_ecl, sizeof(double) * 8 * n_clusters));
        c->h_ecl.resize(8 * (size_t)n_clusters);
        c->h_offsets.assign(offsets, offsets + n_clusters + 1);
        INIT_CUDA(cudaMalloc(&c->d_big, sizeof(int32_t) * n_clusters));
        INIT_CUDA(cudaMalloc(&c->d_small, sizeof(int32_t) * n_clusters));
        INIT_CUDA(cudaMalloc(&c->d_xchg, sizeof(int) * n_clusters));
        INIT_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        INIT_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        INIT_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        INIT_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        {
            const frost_status ts = set_teams(c, kBatchTeamMinN, kBatchTeamBlocks);
            if (ts != FROST_OK) return bail(ts);
        }
    }
    INIT_CUDA(cudaMalloc(&c->dmisc, sizeof(Misc)));
    // the status word of a multi-block single-set solver team (batch contexts have one per cluster)
    if (!c->d_xchg) INIT_CUDA(cudaMalloc(&c->d_xchg, sizeof(int)));
    INIT_CUDA(cudaMallocHost(&c->hmisc, sizeof(Misc)));
    c->main.s = c->stream;
    c->main.recA = c->recA;
    c->main.recB = c->recB;
    c->main.part = c->part;
    c->main.aA = c->aA;
    c->main.aB = c->aB;
    c->main.atA = c->atA;
    c->main.atB = c->atB;
    c->main.wA = c->wA;
    c->main.wB = c->wB;
    c->main.hist = c->hist;
    c->main.hA = c->hA;
    c->main.hB = c->hB;
    c->main.part_hot = c->part_hot;
    c->branch_streams = o.branch_streams >= 0;
    c->sym_cross = o.sym_cross > 0 ? 1 : (o.sym_cross < 0 ? -1 : 0);
    INIT_CUDA(cudaMemsetAsync(c->dmisc, 0, sizeof(Misc), c->stream));
    INIT_CUDA(cudaMemsetAsync(c->marks, 0, sizeof(int32_t) * N, c->stream));
    launch_identity(c->stream, c->all, (int)n);
    // state: [n][3] -> SoA through a scratch copy (inputs may be host or device memory)
    double *tmp = c->aA;
    INIT_CUDA(cudaMemcpyAsync(tmp, x, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
    launch_aos_to_soa(c->stream, tmp, (int)n, c->x, &c->dmisc->err);
    INIT_CUDA(cudaMemcpyAsync(c->aB, v, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
    launch_aos_to_soa(c->stream, c->aB, (int)n, c->v, &c->dmisc->err);
    INIT_CUDA(cudaMemcpyAsync(c->m, m, sizeof(double) * N, cudaMemcpyDefault, c->stream));
    launch_check_mass(c->stream, c->m, (int)n, &c->dmisc->err);
    INIT_CUDA(cudaGetLastError());
    const frost_status st = sync_misc(c);
    if (st != FROST_OK) {
        char why[kLastErrorBytes];
        snprintf(why, sizeof(why), "%s", g_last_error);
        return bail(fail(st, "initial state rejected: %s", why));
    }
#undef INIT_CUDA
    *out = c;
    return FROST_OK;
}

void frost_destroy(frost_ctx *ctx) { destroy(ctx); }

frost_status frost_set_state(frost_ctx *c, const double *x, const double *v, double t)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    const size_t N = (size_t)c->N;
    if (x) {
        FROST_CUDA(cudaMemcpyAsync(c->aA, x, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
        launch_aos_to_soa(c->stream, c->aA, c->N, c->x, &c->dmisc->err);
    }
    if (v) {
        FROST_CUDA(cudaMemcpyAsync(c->aB, v, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
        launch_aos_to_soa(c->stream, c->aB, c->N, c->v, &c->dmisc->err);
    }
    c->t = t;
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_get_state(frost_ctx *c, double *x, double *v, double *t)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    const size_t N = (size_t)c->N;
    if (x) {
        launch_soa_to_aos(c->stream, c->x, c->N, c->aA);
        FROST_CUDA(cudaMemcpyAsync(x, c->aA, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
    }
    if (v) {
        launch_soa_to_aos(c->stream, c->v, c->N, c->aB);
        FROST_CUDA(cudaMemcpyAsync(v, c->aB, sizeof(double) * 3 * N, cudaMemcpyDefault, c->stream));
    }
    if (t) *t = c->t;
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_accel_gradient(frost_ctx *c, const int32_t *active, int64_t n_active,
                                  const int32_t *source, int64_t n_source, double eps_grad,
                                  double *acc, double *acc_tilde, double *grad)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_active, "n_active"));
    FROST_TRY(check_sizes(c, n_source, "n_source"));
    if (!std::isfinite(eps_grad)) return fail(FROST_EINVAL, "eps_grad must be finite");
    const int nA = (int)n_active, nB = (int)n_source;
    const int32_t *A = active ? active : c->all;
    const int32_t *B = source ? source : c->all;
    bool self;
    if (active == source && nA == nB) {
        FROST_TRY(check_list(c, active, nA));
        self = true;
    } else {
        launch_list_relation(c->stream, A, nA, B, nB, c->N, c->marks, c->dmisc->rel);
        FROST_TRY(sync_misc(c));
        if (c->hmisc->rel[0]) return fail(FROST_EINVAL, "index list has an out-of-range or repeated index");
        const int64_t common = c->hmisc->rel[1];
        if (common == nA && nA == nB) self = true;  // the same set in another order
        else if (common == 0) self = false;
        else return fail(FROST_EINVAL, "active and source lists overlap partially (%lld common)", (long long)common);
    }
    if (nA == 0) return FROST_OK;
    const bool want_grad = acc_tilde || grad;
    Lane &M = c->main;
    if (self) {
        unsigned *h = (want_grad && c->mixed) ? zero_hists(M) : nullptr;
        pass_acc(c, M, A, nA, A, nA, true, c->aA, acc, want_grad ? c->wA : nullptr, h);
        if (h) mark_hot(c, M, nA, nA, true, c->aA, h, nullptr, 0, c->hA);
        if (want_grad)
            pass_grad(c, M, A, nA, c->aA, A, nA, c->aA, true, eps_grad, nullptr, acc_tilde, grad, c->wA, c->hA);
    } else if (want_grad && c->mixed && nB > 0 && c->sym_cross >= 0 &&
               (c->sym_cross > 0 || (int64_t)nA * nB >= kSymCrossPrepassMinPairs)) {
        // both accurate passes on records packed once, their prepasses in one symmetric kernel
        unsigned *h = zero_hists(M);
        pack_pos(c, M, A, nA, M.recA);
        pack_pos(c, M, B, nB, M.recB);
        {
            TimedScope ts(c, M.s, PASS_ACC, 0);
            launch_wmax_sym_cross(M.s, M.recA, nA, M.recB, nB, c->eps2, c->n_sm, c->wA, c->wB);
            c->st.kernel_launches += 1;
        }
        pass_acc(c, M, A, nA, B, nB, false, c->aA, acc, c->wA, h, KickArgs(), M.recA, M.recB, true);
        pass_acc(c, M, B, nB, A, nA, false, c->aB, nullptr, c->wB, h + HOT_BINS, KickArgs(), M.recB, M.recA, true);
        mark_hot(c, M, nB, nA, false, c->aB, h + HOT_BINS, h, nA, c->hB);
        pass_grad(c, M, A, nA, c->aA, B, nB, c->aB, false, eps_grad, nullptr, acc_tilde, grad, c->wA, c->hB);
    } else {
        unsigned *h = (want_grad && c->mixed) ? zero_hists(M) : nullptr;
        pass_acc(c, M, A, nA, B, nB, false, c->aA, acc, want_grad ? c->wA : nullptr, h);
        if (want_grad) {
            pass_acc(c, M, B, nB, A, nA, false, c->aB, nullptr, c->wB, h ? h + HOT_BINS : nullptr);
            // only B's accelerations are sources
            if (h) mark_hot(c, M, nB, nA, false, c->aB, h + HOT_BINS, h, nA, c->hB);
            pass_grad(c, M, A, nA, c->aA, B, nB, c->aB, false, eps_grad, nullptr, acc_tilde, grad, c->wA, c->hB);
        }
    }
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_accel_pairwise(frost_ctx *c, const int32_t *a, int64_t n_a, const int32_t *b, int64_t n_b,
                                  double *acc_a, double *acc_b)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_a, "n_a"));
    FROST_TRY(check_sizes(c, n_b, "n_b"));
    const int nA = (int)n_a, nB = (int)n_b;
    const int32_t *A = a ? a : c->all;
    const int32_t *B = b ? b : c->all;
    launch_list_relation(c->stream, A, nA, B, nB, c->N, c->marks, c->dmisc->rel);
    FROST_TRY(sync_misc(c));
    if (c->hmisc->rel[0]) return fail(FROST_EINVAL, "index list has an out-of-range or repeated index");
    if (c->hmisc->rel[1] != 0) return fail(FROST_EINVAL, "the two lists share %lld particles", (long long)c->hmisc->rel[1]);
    Lane &M = c->main;
    if (nA > 0 && nB > 0) {
        pack_pos(c, M, A, nA, M.recA);
        pack_pos(c, M, B, nB, M.recB);
        pass_acc_sym(c, M, A, nA, B, nB, M.aA, M.aB, KickArgs(), KickArgs(), M.recA, M.recB, true);
        if (acc_a) launch_soa_to_aos(c->stream, M.aA, nA, acc_a);
        if (acc_b) launch_soa_to_aos(c->stream, M.aB, nB, acc_b);
    } else {
        if (acc_a && nA > 0) FROST_CUDA(cudaMemsetAsync(acc_a, 0, sizeof(double) * 3 * nA, c->stream));
        if (acc_b && nB > 0) FROST_CUDA(cudaMemsetAsync(acc_b, 0, sizeof(double) * 3 * nB, c->stream));
    }
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_accel_gradient_pairwise(frost_ctx *c, const int32_t *a, int64_t n_a, const int32_t *b,
                                           int64_t n_b, double eps_grad, double *acc_a, double *acc_b,
                                           double *acc_tilde_a, double *acc_tilde_b, double *grad_a, double *grad_b)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_a, "n_a"));
    FROST_TRY(check_sizes(c, n_b, "n_b"));
    const int nA = (int)n_a, nB = (int)n_b;
    const int32_t *A = a ? a : c->all;
    const int32_t *B = b ? b : c->all;
    launch_list_relation(c->stream, A, nA, B, nB, c->N, c->marks, c->dmisc->rel);
    FROST_TRY(sync_misc(c));
    if (c->hmisc->rel[0]) return fail(FROST_EINVAL, "index list has an out-of-range or repeated index");
    if (c->hmisc->rel[1] != 0) return fail(FROST_EINVAL, "the two lists share %lld particles", (long long)c->hmisc->rel[1]);
    Lane &M = c->main;
    if (nA > 0 && nB > 0) {
        pack_pos(c, M, A, nA, M.recA);
        pack_pos(c, M, B, nB, M.recB);
        const bool sym = c->sym_cross >= 0 &&
                         grad_pairwise_sym(c, M, A, nA, B, nB, eps_grad, nullptr, nullptr, acc_tilde_a, acc_tilde_b,
                                           grad_a, grad_b, KickArgs(), KickArgs(), true);
        if (!sym) {
            // two one-sided passes per kind, in the order of kick_sf
            unsigned *h = c->mixed ? zero_hists(M) : nullptr;
            pass_acc(c, M, A, nA, B, nB, false, M.aA, nullptr, M.wA, h, KickArgs(), M.recA, M.recB);
            pass_acc(c, M, B, nB, A, nA, false, M.aB, nullptr, M.wB, h ? h + HOT_BINS : nullptr, KickArgs(), M.recB,
                     M.recA);
            if (h) {
                mark_hot(c, M, nA, nB, false, M.aA, h, h + HOT_BINS, nB, M.hA);
                mark_hot(c, M, nB, nA, false, M.aB, h + HOT_BINS, h, nA, M.hB);
            }
            pack_grad(c, M, A, nA, M.aA, M.recA, c->mixed ? M.hA : nullptr);
            pack_grad(c, M, B, nB, M.aB, M.recB, c->mixed ? M.hB : nullptr);
            pass_grad(c, M, A, nA, M.aA, B, nB, M.aB, false, eps_grad, nullptr, acc_tilde_a, grad_a, M.wA, M.hB,
                      KickArgs(), M.recA, M.recB);
            pass_grad(c, M, B, nB, M.aB, A, nA, M.aA, false, eps_grad, nullptr, acc_tilde_b, grad_b, M.wB, M.hA,
                      KickArgs(), M.recB, M.recA);
        }
        if (acc_a) launch_soa_to_aos(c->stream, M.aA, nA, acc_a);
        if (acc_b) launch_soa_to_aos(c->stream, M.aB, nB, acc_b);
    } else {
        double *outs[] = {acc_a, acc_tilde_a, grad_a};
        for (double *o : outs)
            if (o && nA > 0) FROST_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * 3 * nA, c->stream));
        double *outsb[] = {acc_b, acc_tilde_b, grad_b};
        for (double *o : outsb)
            if (o && nB > 0) FROST_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * 3 * nB, c->stream));
    }
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_timesteps(frost_ctx *c, const int32_t *set, int64_t n_set, double *tau)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_set, "n_set"));
    if (n_set > 0 && !tau) return fail(FROST_EINVAL, "tau is NULL");
    FROST_TRY(check_list(c, set, (int)n_set));
    pass_tstep(c, c->main, set ? set : c->all, (int)n_set, tau);
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_partition(frost_ctx *c, const int32_t *set, int64_t n_set, const double *tau,
                             double tau_pivot, int32_t *S, int32_t *F, int64_t *n_slow, int64_t *n_fast)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_set, "n_set"));
    if (n_set > 0 && (!tau || !S || !F)) return fail(FROST_EINVAL, "tau, S and F are required");
    launch_partition(c->stream, set, (int)n_set, tau, tau_pivot, S, F, c->dmisc->counts, c->pblk);
    c->st.kernel_launches += n_set >= PART_MULTI_MIN ? 2 : 1;
    FROST_CUDA(cudaGetLastError());
    FROST_TRY(sync_misc(c));
    if (n_slow) *n_slow = c->hmisc->counts[0];
    if (n_fast) *n_fast = c->hmisc->counts[1];
    return FROST_OK;
}

frost_status frost_kick(frost_ctx *c, const int32_t *set, int64_t n_set, const double *a, double dt)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_set, "n_set"));
    if (n_set > 0 && !a) return fail(FROST_EINVAL, "a is NULL");
    launch_kick_aos(c->stream, set, (int)n_set, c->v, c->N, a, dt);
    c->st.kernel_launches += (n_set > 0);
    FROST_CUDA(cudaGetLastError());
    return FROST_OK;
}

frost_status frost_drift(frost_ctx *c, const int32_t *set, int64_t n_set, double dt)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_set, "n_set"));
    drift(c, c->main, set, (int)n_set, dt);
    FROST_CUDA(cudaGetLastError());
    return FROST_OK;
}

frost_status frost_fsi(frost_ctx *c, const int32_t *set, int64_t n_set, double dt)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_TRY(check_sizes(c, n_set, "n_set"));
    fsi(c, c->main, set ? set : c->all, (int)n_set, dt);
    FROST_CUDA(cudaGetLastError());
    return FROST_OK;
}

// e^{h H_S}: leapfrog of the set S under its own forces, kick(h/2) drift(h) kick(h/2)
void leapfrog(frost_ctx *c, const int32_t *S, int nS, double h)
{
    if (nS <= 0) return;
    Lane &M = c->main;
    pass_acc(c, M, S, nS, S, nS, true, c->aA, nullptr, nullptr, nullptr, kick_of(c, S, 0.5 * h));
    drift_pack(c, M, S, nS, h, c->recA);
    pass_acc(c, M, S, nS, S, nS, true, c->aA, nullptr, nullptr, nullptr, kick_of(c, S, 0.5 * h), c->recA, c->recA);
}

// The second-order HOLD integrator, Eq. hhs2: e^{eps/2 H_F} e^{eps/2 H_S} e^{eps U_FS}
// e^{eps/2 H_S} e^{eps/2 H_F}, the fast set recursively with the pivot halved.
frost_status hold2(frost_ctx *c, const int32_t *P, int nP, double tau, int depth)
{
    if (nP <= 0) return FROST_OK;
    if (depth > c->max_depth)
        return fail(FROST_EDEPTH, "hold2 deeper than max_depth=%d (|P|=%d, tau_pivot=%g)", c->max_depth, nP, tau);
    c->st.hhs_calls += 1;
    if (depth > c->st.max_depth_seen) c->st.max_depth_seen = depth;
    {
        const int L = std::min(depth, FROST_STATS_LEVELS - 1);
        c->st.level_calls[L] += 1;
        c->st.level_particles[L] += nP;
    }
    FROST_TRY(ensure_level(c, depth));
    int32_t *S = c->lvS[depth], *F = c->lvF[depth];
    pass_tstep(c, c->main, P, nP, c->tau);
    launch_partition(c->stream, P, nP, c->tau, tau, S, F, c->dmisc->counts, c->pblk);
    c->st.kernel_launches += nP >= PART_MULTI_MIN ? 2 : 1;
    FROST_TRY(sync_misc(c));
    const int nS = (int)c->hmisc->counts[0];
    const int nF = (int)c->hmisc->counts[1];
    FROST_TRY(hold2(c, F, nF, 0.5 * tau, depth + 1));
    leapfrog(c, S, nS, 0.5 * tau);
    kick_sf(c, c->main, nullptr, S, nS, F, nF, tau, false, tau);
    leapfrog(c, S, nS, 0.5 * tau);
    return hold2(c, F, nF, 0.5 * tau, depth + 1);
}

// n_steps top-level steps of every cluster of a batch context: one launch per team kind
// (a CUDA graph, captured once per (dt_pivot, n_steps) and replayed)
static frost_status batch_step(frost_ctx *c, double dt_pivot, int64_t n_steps)
{
    // every cluster in its own thread block, all steps in one launch
    if (c->max_depth >= SUBTREE_MAX_FRAMES)
        return fail(FROST_EINVAL, "batch contexts need max_depth < %d", SUBTREE_MAX_FRAMES);
    if (n_steps == 0) return FROST_OK;
    if (n_steps > INT32_MAX) return fail(FROST_EINVAL, "n_steps too large");
    SubtreeArgs a;
    a.x = c->x;
    a.v = c->v;
    a.m = c->m;
    a.N = c->N;
    a.G = c->G;
    a.eta = c->eta;
    a.eps2 = c->eps2;
    a.max_depth = c->max_depth;
    a.err = &c->dmisc->err;
    a.counters = c->dmisc->sub;
    a.levels = &c->dmisc->lev[0][0];
    a.aC = c->aC;
    a.perm = c->perm;
    a.tmp = c->ptmp;
    a.tau = c->tau;
    a.aA = c->aA;
    a.aB = c->aB;
    a.atA = c->atA;
    a.atB = c->atB;
    a.wA = c->wA;
    a.wB = c->wB;
    a.recA = c->recA;
    a.recB = c->recB;
    a.offsets = c->d_offsets;
    a.xchg = c->d_xchg;
    a.overlap = c->branch_streams;
    a.tau0 = dt_pivot;
    a.depth0 = 0;
    a.n_steps = (int)n_steps;
    SubtreeArgs ab = a, as = a;
    ab.cl_index = c->d_big;
    ab.n_teams = c->n_big;
    ab.team_blocks = c->team_blocks;
    as.cl_index = c->d_small;
    as.n_teams = c->n_small;
    if (!c->gexec || c->g_dt != dt_pivot || c->g_steps != n_steps) {
        // capture the step: the large clusters on a forked stream, concurrently with the
        // small ones, joined before the end of the graph
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        FROST_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaSuccess, e2 = cudaSuccess;
        if (c->n_big && c->n_small) {
            cudaEventRecord(c->ev_fork, c->cap);
            cudaStreamWaitEvent(c->side, c->ev_fork, 0);
            e1 = launch_subtree(c->side, c->mixed, c->sym, ab);
            e2 = launch_subtree(c->cap, c->mixed, c->sym, as);
            cudaEventRecord(c->ev_join, c->side);
            cudaStreamWaitEvent(c->cap, c->ev_join, 0);
        } else if (c->n_big) {
            e1 = launch_subtree(c->cap, c->mixed, c->sym, ab);
        } else {
            e2 = launch_subtree(c->cap, c->mixed, c->sym, as);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->cap, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(FROST_ECUDA, "batch step capture: %s",
                        cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : ec)));
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return fail(FROST_ECUDA, "batch step graph: %s", cudaGetErrorString(ei));
        }
        c->g_dt = dt_pivot;
        c->g_steps = n_steps;
    }
    {
        TimedScope ts(c, c->stream, PASS_SUBTREE, 0);
        FROST_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    }
    c->st.kernel_launches += (c->n_big > 0) + (c->n_small > 0);
    c->st.subtree_launches += c->n_clusters;
    c->t += dt_pivot * (double)n_steps;
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_step(frost_ctx *c, double dt_pivot, int64_t n_steps)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (!(dt_pivot > 0.0) || !std::isfinite(dt_pivot)) return fail(FROST_EINVAL, "dt_pivot must be > 0");
    if (n_steps < 0) return fail(FROST_EINVAL, "n_steps < 0");
    if (c->n_clusters > 0) return batch_step(c, dt_pivot, n_steps);
    for (int64_t k = 0; k < n_steps; ++k) {
        if (c->integrator == FROST_HOLD2) FROST_TRY(hold2(c, c->all, c->N, dt_pivot, 0));
        else FROST_TRY(hhs_fsi(c, c->all, c->N, dt_pivot, 0));
        c->t += dt_pivot;
    }
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

// per-cluster sums into c->h_ecl
static frost_status cluster_energies(frost_ctx *c)
{
    launch_cluster_energy(c->stream, c->d_offsets, c->n_clusters, c->x, c->v, c->m, c->N, c->eps2, c->d_ecl);
    c->st.kernel_launches += 1;
    FROST_CUDA(cudaGetLastError());
    FROST_CUDA(cudaMemcpyAsync(c->h_ecl.data(), c->d_ecl, sizeof(double) * 8 * c->n_clusters,
                               cudaMemcpyDeviceToHost, c->stream));
    return sync_misc(c);
}

frost_status frost_energy_clusters(frost_ctx *c, double *E_kin, double *E_pot, double *P, double *L)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (c->n_clusters <= 0) return fail(FROST_EINVAL, "not a batch context");
    FROST_TRY(cluster_energies(c));
    for (int k = 0; k < c->n_clusters; ++k) {
        const double *e = &c->h_ecl[8 * (size_t)k];
        if (E_kin) E_kin[k] = e[0];
        if (E_pot) E_pot[k] = -c->G * e[1];
        for (int q = 0; q < 3; ++q) {
            if (P) P[3 * k + q] = e[2 + q];
            if (L) L[3 * k + q] = e[5 + q];
        }
    }
    return FROST_OK;
}

frost_status frost_energy_momentum(frost_ctx *c, double *E_kin, double *E_pot, double P[3], double L[3])
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (c->n_clusters > 0) {
        FROST_TRY(cluster_energies(c));
        double T = 0.0, W = 0.0, Ps[3] = {0, 0, 0}, Ls[3] = {0, 0, 0};
        for (int k = 0; k < c->n_clusters; ++k) {
            const double *e = &c->h_ecl[8 * (size_t)k];
            T += e[0];
            W += e[1];
            for (int q = 0; q < 3; ++q) {
                Ps[q] += e[2 + q];
                Ls[q] += e[5 + q];
            }
        }
        if (E_kin) *E_kin = T;
        if (E_pot) *E_pot = -c->G * W;
        for (int q = 0; q < 3; ++q) {
            if (P) P[q] = Ps[q];
            if (L) L[q] = Ls[q];
        }
        return FROST_OK;
    }
    // the potential pass skips the tiles below each i-block's diagonal, so its blocks differ in
    // work: eight waves of blocks (of its own occupancy) keep the last ones short
    SplitShape sh;
    {
        const long long cap = (long long)potential_blocks_per_sm() * c->n_sm;
        const int tiles = (int)((c->N + PAIR_TJ - 1) / PAIR_TJ);
        sh.nblk_i = (int)((c->N + PAIR_BS - 1) / PAIR_BS);
        const int ns = (int)std::min<long long>(tiles, std::max<long long>(1, (8 * cap + sh.nblk_i - 1) / sh.nblk_i));
        sh.j_per_split = ((tiles + ns - 1) / ns) * PAIR_TJ;
        sh.nsplit = (int)((c->N + sh.j_per_split - 1) / sh.j_per_split);
    }
    while ((size_t)sh.nsplit * c->N > c->part_elems && sh.nsplit > 1) {
        const int tiles = (c->N + PAIR_TJ - 1) / PAIR_TJ;
        const int ns = std::max(1, sh.nsplit / 2);
        sh.j_per_split = ((tiles + ns - 1) / ns) * PAIR_TJ;
        sh.nsplit = (c->N + sh.j_per_split - 1) / sh.j_per_split;
    }
    launch_potential(c->stream, c->x, c->m, c->N, c->eps2, (float4 *)c->recA, c->part, sh);
    launch_energy_reduce(c->stream, c->x, c->v, c->m, c->N, c->part, sh.nsplit, c->dmisc->eres);
    c->st.kernel_launches += 3;
    FROST_CUDA(cudaGetLastError());
    FROST_TRY(sync_misc(c));
    const double *e = c->hmisc->eres;
    if (E_kin) *E_kin = e[0];
    if (E_pot) *E_pot = -c->G * e[1];  // phi_i sums the pairs j > i
    if (P)
        for (int k = 0; k < 3; ++k) P[k] = e[2 + k];
    if (L)
        for (int k = 0; k < 3; ++k) L[k] = e[5 + k];
    return FROST_OK;
}

frost_status frost_get_stats(frost_ctx *c, frost_stats *out)
{
    if (!c || !out) return fail(FROST_EINVAL, "NULL argument");
    if (c->timing) {
        FROST_CUDA(cudaStreamSynchronize(c->stream));
        resolve_timing(c);
    }
    *out = c->st;
    out->timing_enabled = c->timing ? 1 : 0;
    return FROST_OK;
}

frost_status frost_reset_stats(frost_ctx *c)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (c->timing) {
        FROST_CUDA(cudaStreamSynchronize(c->stream));
        resolve_timing(c);
    }
    c->st = frost_stats{};
    return FROST_OK;
}

frost_status frost_set_timing(frost_ctx *c, int32_t enable)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (c->timing && !enable) {
        FROST_CUDA(cudaStreamSynchronize(c->stream));
        resolve_timing(c);
    }
    c->timing = enable != 0;
    return FROST_OK;
}

// Autotuner of a batch context: the team split (the smallest cluster that gets a team of
// several blocks, and the blocks of such a team), timed as one batch step of every candidate
// from the same saved state; the state and time are restored afterwards.  The step is the
// pivot of the last frost_step call, else 2^-7.
static frost_status batch_autotune(frost_ctx *c, int32_t *out)
{
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    double *sx = nullptr, *sv = nullptr;
    FROST_CUDA(cudaMalloc(&sx, bytes));
    if (cudaMalloc(&sv, bytes) != cudaSuccess) {
        cudaFree(sx);
        return fail(FROST_ENOMEM, "autotune state copy");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double dt = c->g_dt > 0.0 ? c->g_dt : 1.0 / 128.0;
    const double t0 = c->t;
    frost_status st = FROST_OK;
    cudaMemcpyAsync(sx, c->x, bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(sv, c->v, bytes, cudaMemcpyDeviceToDevice, c->stream);
    struct Cand {
        int64_t min_n;
        int blocks;
    };
    std::vector<Cand> cands;
    cands.push_back({INT64_MAX, 1});  // one block per cluster
    for (int64_t mn : {256, 384, 512, 768, 1024, 1536, 2048})
        for (int b : {2, 4, 8}) cands.push_back({mn, b});
    float best = INFINITY;
    Cand pick = {c->team_min_n, c->team_blocks};
    for (const Cand &q : cands) {
        if ((st = set_teams(c, q.min_n, q.blocks)) != FROST_OK) break;
        float tq = INFINITY;
        for (int rep = 0; rep < 3 && st == FROST_OK; ++rep) {
            cudaMemcpyAsync(c->x, sx, bytes, cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(c->v, sv, bytes, cudaMemcpyDeviceToDevice, c->stream);
            // the first call captures the graph of this split; the others replay it
            if (rep > 0) cudaEventRecord(e0, c->stream);
            st = batch_step(c, dt, 1);
            if (st == FROST_OK && rep > 0) {
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tq = std::min(tq, ms);
            }
        }
        if (st != FROST_OK) break;
        if (tq < 0.98f * best) {
            best = tq;
            pick = q;
        }
    }
    cudaMemcpyAsync(c->x, sx, bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->v, sv, bytes, cudaMemcpyDeviceToDevice, c->stream);
    c->t = t0;
    const frost_status st2 = set_teams(c, pick.min_n, pick.blocks);
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sx);
    cudaFree(sv);
    if (st != FROST_OK) return st;
    if (st2 != FROST_OK) return st2;
    if (out) {
        for (int k = 0; k < TUNE_ROWS * 32; ++k) out[k] = 0;
        out[0] = (int32_t)std::min<int64_t>(pick.min_n, INT32_MAX);
        out[1] = pick.blocks;
    }
    return sync_misc(c);
}

frost_status frost_autotune(frost_ctx *c, int32_t *waves_out)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    if (c->n_clusters > 0) return batch_autotune(c, waves_out);
    static const int kWaves[] = {1, 2, 4, 8, 16};
    cudaEvent_t e0, e1;
    FROST_CUDA(cudaEventCreate(&e0));
    FROST_CUDA(cudaEventCreate(&e1));
    for (int k = 9; (1 << k) <= c->N && k < 31; ++k) {
        const int n = 1 << k;
        for (int row = 0; row < (c->mixed ? TUNE_ROWS : 3); ++row) {
            const int kind = (row == TUNE_ACC_ACCURATE) ? PASS_ACC : row;
            const bool accurate = (row == TUNE_ACC_ACCURATE);
            // records of particles 0 .. n-1 (zero accelerations for the gradient records)
            if (kind == PASS_ACC) {
                pack_pos(c, c->main, c->all, n, c->recA);
            } else if (kind == PASS_GRAD) {
                cudaMemsetAsync(c->aB, 0, sizeof(double) * 3 * n, c->stream);
                if (c->mixed) launch_pack_grad_mixed(c->stream, c->all, n, c->x, c->m, c->N, c->aB, (float4 *)c->recA);
                else launch_pack_grad_fp64(c->stream, c->all, n, c->x, c->m, c->N, c->aB, (double4_32a *)c->recA);
            } else {
                const double *acc = nullptr;
                if (c->sym & FROST_FLYBY_EXACT) {
                    cudaMemsetAsync(c->aB, 0, sizeof(double) * 3 * n, c->stream);
                    acc = c->aB;
                }
                if (c->mixed)
                    launch_pack_tstep_mixed(c->stream, c->all, n, c->x, c->v, c->m, c->N, c->G, (float4 *)c->recA,
                                            acc);
                else
                    launch_pack_tstep_fp64(c->stream, c->all, n, c->x, c->v, c->m, c->N, c->G,
                                           (double4_32a *)c->recA, acc);
            }
            // time each distinct launch once (several bounds can give the same one): the
            // 128-record kernels (q < 5) and, in mixed mode, the small-tile ones (q >= 5), each
            // pass with its finalisation, whose cost grows with the number of splits
            const int nq = c->mixed ? 10 : 5;
            float tw[10];
            int splits[10];
            for (int q = 0; q < nq; ++q) {
                PairArgs a;
                a.irec = c->recA;
                a.jrec = c->recA;
                a.n_a = n;
                a.n_s = n;
                a.self_pass = 1;
                a.eps2 = c->eps2;
                a.part = c->part;
                a.shape = shape_for(c, kind, n, n, kWaves[q % 5], q >= 5 ? 1 : 0);
                a.accurate = accurate;
                a.wmax = accurate ? c->wA : nullptr;
                a.jlist = c->all;
                a.m = c->m;
                splits[q] = a.shape.nsplit;
                tw[q] = INFINITY;
                for (int r = (q / 5) * 5; r < q; ++r)
                    if (splits[r] == splits[q]) tw[q] = tw[r];
                if (tw[q] < INFINITY) continue;
                for (int rep = 0; rep < 4; ++rep) {
                    cudaEventRecord(e0, c->stream);
                    if (accurate) launch_wmax(c->stream, a, c->wA);
                    if (kind == PASS_ACC) launch_acc(c->stream, c->mixed, a);
                    else if (kind == PASS_GRAD) launch_grad(c->stream, c->mixed, a);
                    else launch_tstep(c->stream, c->mixed, a, c->eta, c->sym, &c->dmisc->err);
                    if (kind == PASS_TSTEP)
                        launch_finalize_tau(c->stream, c->part, a.shape.nsplit, n, c->eta, c->aB, &c->dmisc->err);
                    else
                        launch_finalize_vec(c->stream, c->part, a.shape.nsplit, n, 1.0, c->aB, nullptr,
                                            &c->dmisc->err, 0);
                    cudaEventRecord(e1, c->stream);
                    FROST_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tw[q] = std::min(tw[q], ms);  // the first launch warms the caches
                }
            }
            // the fastest launch, if it beats the default (8 waves, the default kernel
            // choice) by 3%; negative entries select the small-tile kernels
            const int q0 = shape_for(c, kind, n, n, 8).small ? 8 : 3;
            int best_q = q0;
            float best = tw[q0];
            for (int q = 0; q < nq; ++q)
                if (tw[q] < 0.97f * tw[q0] && tw[q] < best) {
                    best = tw[q];
                    best_q = q;
                }
            c->tune_w[row][k] = (best_q >= 5) ? -kWaves[best_q % 5] : kWaves[best_q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (waves_out)
        for (int q = 0; q < TUNE_ROWS; ++q)
            for (int k = 0; k < 32; ++k) waves_out[q * 32 + k] = c->tune_w[q][k];
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_synchronize(frost_ctx *c)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_CUDA(cudaGetLastError());
    return sync_misc(c);
}

frost_status frost_clear_error(frost_ctx *c)
{
    if (!c) return fail(FROST_EINVAL, "NULL context");
    FROST_CUDA(cudaMemsetAsync(&c->dmisc->err, 0, sizeof(int), c->stream));
    FROST_CUDA(cudaStreamSynchronize(c->stream));
    clear_last_error();
    return FROST_OK;
}

}  // extern "C"
