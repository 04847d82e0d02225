// Internal declarations of the sm_103a HHS-FSI kernels (not part of the C-ABI).
//
// Device data layout (all owned by a frost_ctx):
//   x, v : FP64 structure of arrays, component c of particle i at [c * N + i]
//   m    : FP64 masses [N]
// Every pair pass works on packed, contiguous per-pass records of its active list A and its
// source list B (built by the pack kernels from the SoA store and the index lists), so the
// pair kernels stream their j-tiles linearly through shared memory.
//
// Mixed-precision records (FP32, 16-byte aligned float4):
//   acc / time-step pass:  p0 = {x_hi, y_hi, z_hi, m}, p1 = {x_lo, y_lo, z_lo, 0}
//                          with x_hi = fp32(x), x_lo = fp32(x - x_hi)  (float-float, 48 bits)
//                          time-step pass adds pv = {vx, vy, vz, G m}
//   gradient pass:         q0 = {x_h, y_h, z_h, m}, q1 = {x_m, y_m, z_m, ah_x},
//                          q2 = {x_l, y_l, z_l, ah_y}, q3 = {ah_z, al_x, al_y, al_z}
//                          x = x_h + x_m + x_l with x_h, x_m holding 12 significant bits, so
//                          ((x_hj - x_hi) + (x_mj - x_mi)) is exact and the separation is
//                          rounded once; a = ah + al with ah holding 12 significant bits.
// FP64 records: d0 = {x, y, z, m}, d1 = {ax, ay, az, 0} (gradient), dv = {vx, vy, vz, G m}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace frost {

// Message of the last failure in the calling host thread, returned by frost_last_error();
// kept in fixed thread-local storage (formatting it allocates nothing).
constexpr int kLastErrorBytes = 512;
void set_last_error(const char *fmt, ...) __attribute__((format(printf, 1, 2)));
void clear_last_error();

// device error word bits
enum : int {
    ERR_NONFINITE = 1 << 0,
    ERR_COINCIDENT = 1 << 1,
    ERR_INDEX = 1 << 2,
    ERR_TIMEOUT = 1 << 3,
    ERR_DUPLICATE = 1 << 4,
    ERR_DEPTH = 1 << 5,
};

// kinds of timed kernels (the subtree solver runs all passes of a small set)
enum PassKind { PASS_ACC = 0, PASS_GRAD = 1, PASS_TSTEP = 2, PASS_SUBTREE = 3 };

// Tile geometry of the pair kernels.
constexpr int PAIR_BS = 128;   // threads per block
constexpr int PAIR_ILP = 2;    // i-particles per thread (mixed)
constexpr int PAIR_TJ = 128;   // j-records per shared-memory tile
constexpr int PAIR_ILP64 = 1;  // i-particles per thread (FP64)
// small-tile instantiation of the mixed pair kernels: one warp a block, tiles of 32 sources;
// spreads the passes of a few hundred particles over all SMs, where the 128-record layout
// leaves most SMs idle and the rest latency-bound
constexpr int PAIR_BS_SMALL = 32;
constexpr int PAIR_TJ_SMALL = 32;

struct SplitShape {
    int nblk_i;       // blocks along the active list
    int nsplit;       // blocks along the source list (j-split)
    int j_per_split;  // sources per split (multiple of the tile size)
    int small = 0;    // 1: the small-tile kernels (PAIR_BS_SMALL, PAIR_TJ_SMALL; mixed only)
};

struct PairArgs {
    // records of the active list (i) and of the source list (j)
    const void *irec;
    const void *jrec;
    int n_a, n_s;
    int self_pass;    // 1 if the two lists are the same list (same positions)
    double eps2;      // softening^2
    double *part;     // partial results [nsplit][ncomp][n_a]
    SplitShape shape;
    const float *wmax = nullptr;   // grad and accurate acc (mixed): max_j m_j / r^3 [n_a], or NULL
    bool accurate = false;         // acc (mixed): the variant that feeds a gradient pass (wmax set)
    const int32_t *jlist = nullptr;  // accurate acc: the source list (NULL: identity) and the
    const double *m = nullptr;       // FP64 masses of the store, for the double-float terms
};

// ---- pack kernels: list -> per-pass records ------------------------------------------
void launch_pack_pos_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                           const double *m, int N, float4 *rec);
// hot (optional): mask bit k set zeroes the mass of record k (a source summed in double-float)
void launch_pack_grad_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                            const double *m, int N, const double *acc /*[3][n]*/, float4 *rec,
                            const uint32_t *hot = nullptr);
// acc (optional, [3][n] by list position): the set's accelerations, packed for the exact
// fly-by derivative (record 3 mixed, record 2 FP64)
void launch_pack_tstep_mixed(cudaStream_t s, const int32_t *list, int n, const double *x,
                             const double *v, const double *m, int N, double G, float4 *rec,
                             const double *acc = nullptr);
void launch_pack_pos_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                          const double *m, int N, double4_32a *rec);
void launch_pack_grad_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                           const double *m, int N, const double *acc, double4_32a *rec);
void launch_pack_tstep_fp64(cudaStream_t s, const int32_t *list, int n, const double *x,
                            const double *v, const double *m, int N, double G, double4_32a *rec,
                            const double *acc = nullptr);

// ---- pair kernels ---------------------------------------------------------------------
// acc: part[split][c][i] = sum_j m_j x_ji / r^3 over the split's sources
// accurate mixed variant (a.accurate): the terms above wmax / 16 (a.wmax from launch_wmax
// at the same records) are summed in double-float
void launch_acc(cudaStream_t s, bool mixed, const PairArgs &a);
// mixed prepass of the accurate Newtonian pass: wmax[i] = max_j m_j / r^3 (zeroed here)
void launch_wmax(cudaStream_t s, const PairArgs &a, float *wmax);
// grad: part[split][c][i] = sum_j m_j r^-5 (r^2 a_ji - 3 (x_ji . a_ji) x_ji)
void launch_grad(cudaStream_t s, bool mixed, const PairArgs &a);
// time-step: part[split][i] = min_j min(t_ff s(eta dt_ff), t_fb s(eta dt_fb)) (without eta)
void launch_tstep(cudaStream_t s, bool mixed, const PairArgs &a, double eta, int sym, int *err);

// ---- finalisation of split partials ---------------------------------------------------
// Optional kick fused into a finalisation: v[c][list[i]] += dt * (the value written for i),
// with the separate roundings of launch_kick (v = NULL: no kick; list = NULL: identity);
// store (optional): the value is also written to store[c][list[i]] ([3][N], by particle).
struct KickArgs {
    const int32_t *list = nullptr;
    double *v = nullptr;
    int N = 0;
    double dt = 0.0;
    double *store = nullptr;
};

// out_soa[c][i] = scale * sum_split part[split][c][i]  (also [i][3] copy if out_aos != NULL),
// then the kick / store of kick
void launch_finalize_vec(cudaStream_t s, const double *part, int nsplit, int n, double scale,
                         double *out_soa, double *out_aos, int *err, int coincident_bit,
                         KickArgs kick = KickArgs());
// a~ = a + c g with g = scale * (sum part + sum part2); writes a~ (soa and/or aos) and g
// (aos, optional); part2 (nsplit2 splits, may be 0) holds the double-float terms of hot sources
void launch_finalize_grad(cudaStream_t s, const double *part, int nsplit, int n, double scale,
                          const double *a_soa, double c, double *at_soa, double *at_aos,
                          double *g_aos, int *err, int coincident_bit,
                          const double *part2 = nullptr, int nsplit2 = 0, KickArgs kick = KickArgs());

// ---- hot sources of the mixed gradient pass (hot_kernels.cu) -------------------------
constexpr int HOT_BINS = 1024;          // |a| histogram: 4 bins per octave
constexpr float HOT_KAPPA = 6.0f;       // hot: |a| > HOT_KAPPA x (median bin's upper edge)
constexpr int HOT_MAX_SPLITS = 16;      // source splits of k_grad_hot
// hist[HOT_BINS] += counts of the bins of |a_i| over [3][n] accelerations (hist pre-zeroed)
void launch_acc_hist(cudaStream_t s, const double *a_soa, int n, unsigned *hist);
// after an accurate mixed Newtonian pass of A against B (a_soa [3][n_a]): writes the hot
// mask of A (words [(n_a + 31) / 32]).  hist: the |a| histogram of this pass; hist2 (n2
// values): that of the pass of B against A in a cross pair, or NULL.
void launch_hot_mask(cudaStream_t s, const double *a_soa, int n_a, const unsigned *hist,
                     const unsigned *hist2, int n2, uint32_t *mask);
// number of source splits of launch_grad_hot for these list sizes
int hot_grad_splits(int n_a, int n_s, int n_sm);
// part[s][c][i] = FP64 gradient sums over the hot sources of B (mask) for every i of A
void launch_grad_hot(cudaStream_t s, const int32_t *A, int n_a, const double *aA, const int32_t *B,
                     int n_s, const double *aB, const uint32_t *mask, int self_pass, const double *x,
                     const double *m, int N, double eps2, int nsplit, double *part);
// tau[i] = eta * min_split part[split][i]; flags non-positive or NaN values
void launch_finalize_tau(cudaStream_t s, const double *part, int nsplit, int n, double eta,
                         double *tau, int *err);

// ---- integrator kernels ---------------------------------------------------------------
void launch_kick(cudaStream_t s, const int32_t *list, int n, double *v, int N,
                 const double *a_soa, double dt);
void launch_kick_aos(cudaStream_t s, const int32_t *list, int n, double *v, int N,
                     const double *a_aos, double dt);
// v[c][list[k]] += dt * a_glob[c][list[k]]  (accelerations stored by particle, [3][N])
void launch_kick_by_particle(cudaStream_t s, const int32_t *list, int n, double *v, int N,
                             const double *a_glob, double dt);
void launch_drift(cudaStream_t s, const int32_t *list, int n, double *x, const double *v,
                  int N, double dt);
// drift, then pack the moved particles' position records for the next Newtonian pass:
// mode 0 mixed {hi, lo} records, 2 FP64
void launch_drift_pack(cudaStream_t s, const int32_t *list, int n, double *x, const double *v,
                       const double *m, int N, double dt, void *rec, int mode);
// stable partition: S gets set[k] with tau[k] >= pivot, F the rest; counts[0] = |S|,
// counts[1] = |F|
// stable slow / fast split (tau >= pivot first, both in list order); counts = {|S|, |F|}.  With
// blk (int scratch of partition_blocks(n)) and n >= PART_MULTI_MIN, many blocks (two launches)
// instead of one; the lists are the same.
constexpr int PART_MULTI_MIN = 8192;
inline int partition_blocks(int n) { return (n + 4095) / 4096; }
void launch_partition(cudaStream_t s, const int32_t *set, int n, const double *tau,
                      double pivot, int32_t *S, int32_t *F, int64_t *counts, int *blk = nullptr);

// ---- validation and reductions --------------------------------------------------------
// marks[] (int32[N]) must be zero on entry and is returned to zero on exit.
// out[0] = bad index or repeated index in either list (0/1), out[1] = |A cap B|
void launch_list_relation(cudaStream_t s, const int32_t *A, int nA, const int32_t *B, int nB,
                          int N, int32_t *marks, int64_t *out);
void launch_check_finite(cudaStream_t s, const double *p, int64_t n, int *err);
void launch_identity(cudaStream_t s, int32_t *list, int n);
// [n][3] -> [3][n] (flags non-finite values) and back; masses must be finite and > 0
void launch_aos_to_soa(cudaStream_t s, const double *aos, int n, double *soa, int *err);
void launch_soa_to_aos(cudaStream_t s, const double *soa, int n, double *aos);
void launch_check_mass(cudaStream_t s, const double *m, int n, int *err);
// phi_i = sum_{j > i} m_j / sqrt(r^2 + eps2) (each pair once; U = -G sum_i m_i phi_i) in double-float
// arithmetic (about 1e-13 relative), split partials part[split][i] (summed in order by
// launch_energy_reduce); rec: scratch of 48 B per particle
void launch_potential(cudaStream_t s, const double *x, const double *m, int n, double eps2, float4 *rec,
                      double *part, const SplitShape &shape);
// blocks of the potential pass per SM (its occupancy)
int potential_blocks_per_sm();
// out[0] = T, out[1] = sum_i m_i phi_i, out[2..4] = P, out[5..7] = L (one block, fixed order)
void launch_energy_reduce(cudaStream_t s, const double *x, const double *v, const double *m,
                          int N, const double *part, int nsplit, double *out);
// per-cluster {T, sum_{i<j} m_i m_j / r, P, L} into out[n_clusters][8] (one block per cluster)
void launch_cluster_energy(cudaStream_t s, const int64_t *offsets, int n_clusters, const double *x,
                           const double *v, const double *m, int N, double eps2, double *out);

// ---- symmetric inter-level Newtonian pass (sym_kernels.cu) -------------------------------
// Every pair of two disjoint lists A (n_a) and B (n_s) once: part[split][c][i] = sum over the
// split's sources of m_j x_ji / r^3 (as launch_acc), pj[group][c][j] = sum over the group's
// i-blocks of m_i x_ji / r^3 (the force on j is -G times the sum over the groups).
struct SymShape {
    int nblk_i = 1;        // i-blocks of A
    int ngroups = 1;       // blocks along A (each takes every ngroups-th i-block)
    int nsplit = 1;        // blocks along B
    int j_per_split = 0;   // sources per split (a multiple of the tile)
    int blocks_per_wave = 1;
    long long max_blocks = 1;  // the largest grid the lists allow (one tile per split)
};
// the symmetric cross kernels (their occupancies differ)
enum { SYM_ACC_MIXED = 0, SYM_ACC_FP64 = 1, SYM_ACC_DEFER = 2, SYM_GRAD = 3, SYM_KINDS = 4 };
// part_elems / pj_elems: the capacities of part and pj in doubles
SymShape sym_shape(int kind, int n_a, int n_s, int n_sm, size_t part_elems, size_t pj_elems);
void launch_acc_sym(cudaStream_t s, bool mixed, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                    double *part, double *pj, const SymShape &sh);

// Symmetric passes of the gradient kick_sf (mixed): both lists' accurate Newtonian sums with
// their dominant terms in double-float (wA, wB: max_j m_j / r^3 of each list against the other;
// ilist, jlist: the lists' particle indices for the FP64 masses mstore, NULL = identity), then
// both gradients (records of launch_pack_grad_mixed, hot sources with zero mass).  part: the
// A side per split as launch_acc / launch_grad; pj: the B side per group with the receiver's
// sign (sum_i of the terms of j due to i).
// pcnt: [ngroups][SYM_PCNT_WARPS][n_s] bytes of scratch (the B side's slot counts).
constexpr int SYM_PCNT_WARPS = 4;
void launch_acc_sym_defer(cudaStream_t s, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                          const float *wA, const float *wB, const int32_t *ilist, const int32_t *jlist,
                          const double *mstore, double *part, double *pj, uint8_t *pcnt, const SymShape &sh);
void launch_grad_sym(cudaStream_t s, const void *irec, const void *jrec, int n_a, int n_s, double eps2,
                     const float *wA, const float *wB, double *part, double *pj, uint8_t *pcnt, const SymShape &sh);

// Symmetric time-step pass over one set (mixed): every pair once, tau[i] written directly.
// jbest: [n] unsigned scratch (the j-side minima as FP32 bits); part: [blocks of row 0][n].
struct TstepSymShape {
    int ntiles = 0;  // 128-record tiles of the set
    int tps = 1;     // tiles per split of a row
    int blocks = 0;  // blocks of the upper triangle
};
TstepSymShape tstep_sym_shape(int n, int n_sm, size_t part_elems);
void launch_tstep_sym(cudaStream_t s, const void *rec, int n, double eta, int sym, const TstepSymShape &sh,
                      double *part, unsigned *jbest, double *tau, int *err);

// Symmetric prepasses of the Newtonian pass that feeds a gradient (mixed): wmax = max_j m_j / r^3
// for one set (every pair once), or for two disjoint lists at once (wA, wB); zeroed here.
void launch_wmax_sym_self(cudaStream_t s, const void *rec, int n, double eps2, int n_sm, size_t part_elems,
                          float *wmax);
void launch_wmax_sym_cross(cudaStream_t s, const void *recA, int nA, const void *recB, int nB, double eps2, int n_sm,
                           float *wA, float *wB);

// ---- single-CTA subtree solver (subtree.cu) ------------------------------------------
constexpr int SUBTREE_MAX_FRAMES = 64;  // recursion frames per block (max_depth < 64)
constexpr int SUBTREE_STAT_LEVELS = 48; // per-depth statistics (last entry: deeper levels)
constexpr int SUBTREE_MAX_CLUSTER = 8;  // blocks per team at most (portable cluster size)

struct SubtreeArgs {
    double *x, *v;
    const double *m;
    int N;
    double G, eta, eps2;
    int max_depth;
    int *err;
    unsigned long long *counters;  // [8]: acc, grad, tstep pairs, hhs calls, fsi calls, max depth,
                                   // reused acc pairs, fsi calls run beside the warp path
    unsigned long long *levels;    // [2][SUBTREE_STAT_LEVELS]: calls and set sizes per depth
    double *aC;                    // [3][N] by particle: a^SS kept from the first fsi(S) to the second
    // workspace (per particle: perm, tmp int32; tau double; aA..atB [3] doubles; wA, wB
    // float; recA, recB 64 bytes), indexed from the block's first particle
    int32_t *perm, *tmp;
    double *tau, *aA, *aB, *atA, *atB;
    float *wA, *wB;
    void *recA, *recB;
    // single-set mode: list P of n particles; batch mode: offsets[n_clusters + 1] and, for the
    // n_teams teams of this launch, the cluster of each team (cl_index, or NULL: team t takes
    // cluster t)
    const int32_t *P = nullptr;
    int n = 0;
    const int64_t *offsets = nullptr;
    const int32_t *cl_index = nullptr;
    int n_teams = 0;
    // blocks per team: 1, or a thread-block cluster of 2..SUBTREE_MAX_CLUSTER blocks that
    // share one set; xchg: one int per team (a status word between the team's blocks)
    int team_blocks = 1;
    int *xchg = nullptr;
    // one-block teams: the FSI steps of a slow set on warps 1..7 beside warp 0's subtree of a
    // fast set of at most 32 particles (same results as the serial order)
    bool overlap = false;
    double tau0;
    int depth0;
    int n_steps;
};
cudaError_t launch_subtree(cudaStream_t s, bool mixed, int sym, const SubtreeArgs &a);

// max_waves: at most this many full waves of blocks (the autotuner picks it per size)
SplitShape choose_shape(int n_a, int n_s, int i_per_block, int blocks_per_sm, int n_sm, int max_waves = 8,
                        int tj = PAIR_TJ);
int pair_blocks_per_sm(int kind, bool mixed, bool small = false);
int pair_i_per_block(bool mixed);

}  // namespace frost
