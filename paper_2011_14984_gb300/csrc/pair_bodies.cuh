// Device code shared by the grid pair kernels (pair_kernels.cu) and the single-CTA
// subtree solver (subtree.cu): record builders, pair bodies and per-i-block loops of the
//   Newtonian pass     a_i = G sum_j m_j x_ji / r_ji^3                        (Eq. acc-newton)
//   gradient pass      g_i = 2G sum_j m_j r^-5 (r^2 a_ji - 3 (x_ji . a_ji) x_ji) (Eq. acc-gradient-g)
//   time-step pass     tau_i = eta min_j min(t_ff s(d_ff), t_fb s(d_fb))       (Sec. 4)
// in mixed precision (FP32 bodies on float-float separations, compensated sums) and FP64.
// The record layouts are described in frost_internal.cuh.
#pragma once

#include "df_arith.cuh"
#include "frost_internal.cuh"

#include <cfloat>
#include <cmath>
#include <type_traits>

namespace frost {
namespace dev {

__device__ __forceinline__ void fold2(float &hi, float &lo, float p)
{
    // TwoSum (Knuth): hi + p = s + e exactly
    const float s = hi + p;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += e;
}

__device__ __forceinline__ float trunc12(float f)
{
    // keep sign, exponent and the 11 leading fraction bits (12 significant bits)
    return __uint_as_float(__float_as_uint(f) & 0xFFFFF800u);
}

__device__ __forceinline__ void split3(double p, float &h, float &mi, float &l)
{
    double r = p;
    h = trunc12((float)r);
    r -= (double)h;   // exact
    mi = trunc12((float)r);
    r -= (double)mi;  // exact
    l = (float)r;
}


// ======================================================================================
// Per-particle record builders (one list entry k); used by the pack kernels and by the
// subtree solver's block-wide packs.
// ======================================================================================
__device__ __forceinline__ void pack_pos_mixed_one(int k, const int32_t *__restrict__ list, int n,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ m, int N,
                                                   float4 *__restrict__ rec)
{
    const int i = list ? list[k] : k;
    const double px = x[i], py = x[N + i], pz = x[2 * N + i];
    const float hx = (float)px, hy = (float)py, hz = (float)pz;
    const double mi = m[i];
    const float mh = (float)mi;
    rec[k] = make_float4(hx, hy, hz, mh);
    // the low part of the mass completes its double-float (the dominant terms' weights)
    rec[n + k] = make_float4((float)(px - (double)hx), (float)(py - (double)hy),
                             (float)(pz - (double)hz), (float)(mi - (double)mh));
}

// acc may be NULL (positions only, for the Newtonian pass that precedes the gradient)
__device__ __forceinline__ void pack_grad_mixed_one(int k, const int32_t *__restrict__ list, int n,
                                                    const double *__restrict__ x,
                                                    const double *__restrict__ m, int N,
                                                    const double *__restrict__ acc,
                                                    float4 *__restrict__ rec,
                                                    const uint32_t *__restrict__ hot = nullptr)
{
    const int i = list ? list[k] : k;
    const bool zero_m = hot && ((hot[k >> 5] >> (k & 31)) & 1u);
    float hx, hy, hz, mx, my, mz, lx, ly, lz;
    split3(x[i], hx, mx, lx);
    split3(x[N + i], hy, my, ly);
    split3(x[2 * N + i], hz, mz, lz);
    const double ax = acc ? acc[k] : 0.0, ay = acc ? acc[n + k] : 0.0, az = acc ? acc[2 * n + k] : 0.0;
    const float ahx = trunc12((float)ax), ahy = trunc12((float)ay), ahz = trunc12((float)az);
    rec[k] = make_float4(hx, hy, hz, zero_m ? 0.f : (float)m[i]);
    rec[n + k] = make_float4(mx, my, mz, ahx);
    rec[2 * n + k] = make_float4(lx, ly, lz, ahy);
    rec[3 * n + k] = make_float4(ahz, (float)(ax - (double)ahx), (float)(ay - (double)ahy),
                                 (float)(az - (double)ahz));
}

__device__ __forceinline__ void pack_tstep_mixed_one(int k, const int32_t *__restrict__ list, int n,
                                                     const double *__restrict__ x,
                                                     const double *__restrict__ v,
                                                     const double *__restrict__ m, int N, double G,
                                                     float4 *__restrict__ rec,
                                                     const double *__restrict__ acc = nullptr)
{
    const int i = list ? list[k] : k;
    const double px = x[i], py = x[N + i], pz = x[2 * N + i];
    const float hx = (float)px, hy = (float)py, hz = (float)pz;
    rec[k] = make_float4(hx, hy, hz, (float)m[i]);
    rec[n + k] = make_float4((float)(px - (double)hx), (float)(py - (double)hy),
                             (float)(pz - (double)hz), 0.f);
    rec[2 * n + k] = make_float4((float)v[i], (float)v[N + i], (float)v[2 * N + i],
                                 (float)(G * m[i]));
    // exact fly-by derivative: the accelerations of the set ([3][n], by list position)
    if (acc) rec[3 * n + k] = make_float4((float)acc[k], (float)acc[n + k], (float)acc[2 * n + k], 0.f);
}

__device__ __forceinline__ void pack_pos_fp64_one(int k, const int32_t *__restrict__ list, int n,
                                                  const double *__restrict__ x,
                                                  const double *__restrict__ m, int N,
                                                  double4_32a *__restrict__ rec)
{
    const int i = list ? list[k] : k;
    rec[k] = make_double4_32a(x[i], x[N + i], x[2 * N + i], m[i]);
}

__device__ __forceinline__ void pack_grad_fp64_one(int k, const int32_t *__restrict__ list, int n,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ m, int N,
                                                   const double *__restrict__ acc,
                                                   double4_32a *__restrict__ rec)
{
    const int i = list ? list[k] : k;
    rec[k] = make_double4_32a(x[i], x[N + i], x[2 * N + i], m[i]);
    rec[n + k] = make_double4_32a(acc[k], acc[n + k], acc[2 * n + k], 0.0);
}

__device__ __forceinline__ void pack_tstep_fp64_one(int k, const int32_t *__restrict__ list, int n,
                                                    const double *__restrict__ x,
                                                    const double *__restrict__ v,
                                                    const double *__restrict__ m, int N, double G,
                                                    double4_32a *__restrict__ rec,
                                                    const double *__restrict__ acc = nullptr)
{
    const int i = list ? list[k] : k;
    rec[k] = make_double4_32a(x[i], x[N + i], x[2 * N + i], m[i]);
    rec[n + k] = make_double4_32a(v[i], v[N + i], v[2 * N + i], G * m[i]);
    if (acc) rec[2 * n + k] = make_double4_32a(acc[k], acc[n + k], acc[2 * n + k], 0.0);
}
// Dominant terms.  A term with m_j / r^3 above SLOT_FRACTION x max_j m_j / r^3 is kept out
// of the FP32 partial sums (a heavy term sets the rounding of every later addition to its
// partial sum) and up to GRAD_SLOTS of them per particle are evaluated in double-float after
// the loop.  The j indices wait in registers (constant slot indices after unrolling).
constexpr int GRAD_SLOTS = 8;
constexpr float SLOT_FRACTION = 0.0625f;

template <int ILP>
struct BigSlots;
template <int ILP>
__device__ __forceinline__ void push_big(BigSlots<ILP> &b, int k, int j);

// slot indices in registers (the single-CTA solver's bodies)
template <int ILP>
struct BigSlots {
    int n[ILP];
    int j[GRAD_SLOTS][ILP];
    __device__ __forceinline__ bool room(int k) const { return n[k] < GRAD_SLOTS; }
    __device__ __forceinline__ void push(int k, int jj) { push_big(*this, k, jj); }
    __device__ __forceinline__ int get(int s, int k) const { return j[s][k]; }
};

// slot indices in shared memory, one column per thread (the grid kernels: saves the
// 2 x GRAD_SLOTS registers that would cost occupancy); row (s * ILP + k) of STRIDE words
template <int ILP, int STRIDE>
struct SmemSlots {
    int n[ILP];
    int *col;
    __device__ __forceinline__ bool room(int k) const { return n[k] < GRAD_SLOTS; }
    __device__ __forceinline__ void push(int k, int jj) { col[(n[k] * ILP + k) * STRIDE] = jj; ++n[k]; }
    __device__ __forceinline__ int get(int s, int k) const { return col[(s * ILP + k) * STRIDE]; }
};

template <int ILP>
__device__ __forceinline__ void init_big(BigSlots<ILP> &b, int fill)
{
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        b.n[k] = 0;
#pragma unroll
        for (int s = 0; s < GRAD_SLOTS; ++s) b.j[s][k] = fill;
    }
}

template <int ILP>
__device__ __forceinline__ void push_big(BigSlots<ILP> &b, int k, int j)
{
    const int c = b.n[k];
#pragma unroll
    for (int s = 0; s < GRAD_SLOTS; ++s)
        if (s == c) b.j[s][k] = j;
    b.n[k] = c + 1;
}

struct D3 {
    double x, y, z;
};

// The deferred double-float terms of a one-warp block, evaluated by all its lanes.
// The items (k, s, lane) with s < n[k] of that lane are numbered in that order; lane l
// evaluates items l, l + 32, ... (term(owner lane, k, s) returns the term), and every owner
// then adds its own terms to acc[k] in slot order.  The additions, and so the sums, are those
// of a per-thread loop over the slots, bit for bit; the per-thread loop runs as many rounds
// as the warp's busiest lane has slots, with most lanes idle.  xbuf: 32 D3 of shared memory
// for the warp.
template <int ILP, class Term>
__device__ __forceinline__ void warp_slot_terms(const int (&n)[ILP], D3 *xbuf, double (&acc)[ILP][3], Term term)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    unsigned mask[ILP][GRAD_SLOTS];
    int first[ILP][GRAD_SLOTS];
    int total = 0;
#pragma unroll
    for (int k = 0; k < ILP; ++k)
#pragma unroll
        for (int s = 0; s < GRAD_SLOTS; ++s) {
            mask[k][s] = __ballot_sync(0xffffffffu, s < n[k]);
            first[k][s] = total;
            total += __popc(mask[k][s]);
        }
    for (int base = 0; base < total; base += 32) {
        const int q = base + (int)lane;
        D3 t = {0.0, 0.0, 0.0};
        if (q < total) {
            // the group (k, s) that holds item q, and its owner: the (q - first)-th lane of the group
            int gk = 0, gs = 0;
#pragma unroll
            for (int k = 0; k < ILP; ++k)
#pragma unroll
                for (int s = 0; s < GRAD_SLOTS; ++s)
                    if (mask[k][s] != 0u && first[k][s] <= q) {
                        gk = k;
                        gs = s;
                    }
            unsigned mk = 0u;
            int r = 0;
#pragma unroll
            for (int k = 0; k < ILP; ++k)
#pragma unroll
                for (int s = 0; s < GRAD_SLOTS; ++s)
                    if (k == gk && s == gs) {
                        mk = mask[k][s];
                        r = q - first[k][s];
                    }
            for (; r > 0; --r) mk &= mk - 1u;
            t = term(__ffs(mk) - 1, gk, gs);
        }
        xbuf[lane] = t;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < ILP; ++k)
#pragma unroll
            for (int s = 0; s < GRAD_SLOTS; ++s)
                if (s < n[k]) {
                    const int qo = first[k][s] + __popc(mask[k][s] & below) - base;
                    if (qo >= 0 && qo < 32) {
                        acc[k][0] += xbuf[qo].x;
                        acc[k][1] += xbuf[qo].y;
                        acc[k][2] += xbuf[qo].z;
                    }
                }
        __syncwarp();
    }
}

// The Newtonian pair term of acc_term_df in FP64, from the same records, for a pair whose
// double-float evaluation leaves the FP32 exponent range (r^-3 above ~3e38, r below ~1e-13)
static __device__ __noinline__ D3 acc_term_fp64(const float4 J0, const float4 J1, float ixh, float iyh, float izh,
                                                float ixl, float iyl, float izl, double mj, double eps2)
{
    const double dx = ((double)J0.x + (double)J1.x) - ((double)ixh + (double)ixl);
    const double dy = ((double)J0.y + (double)J1.y) - ((double)iyh + (double)iyl);
    const double dz = ((double)J0.z + (double)J1.z) - ((double)izh + (double)izl);
    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
    const double ri = 1.0 / sqrt(r2);
    const double w = mj * ri * ri * ri;
    D3 r;
    r.x = w * dx;
    r.y = w * dy;
    r.z = w * dz;
    return r;
}

// One Newtonian pair term m_j x_ji / r^3 in double-float from the float-float position
// records (positions to 48 bits) and the FP64 mass mj (the two partners of a tight pair then
// carry exactly opposite momenta, which the gradients of the other particles difference).
// A term outside the FP32 exponent range is evaluated in FP64 instead.
static __device__ __noinline__ D3 acc_term_df(const float4 J0, const float4 J1, float ixh, float iyh, float izh,
                                              float ixl, float iyl, float izl, double mj, double eps2)
{
    using df::dfloat;
    const dfloat dx = df::sub(df::make(J0.x, J1.x), df::make(ixh, ixl));
    const dfloat dy = df::sub(df::make(J0.y, J1.y), df::make(iyh, iyl));
    const dfloat dz = df::sub(df::make(J0.z, J1.z), df::make(izh, izl));
    const dfloat r2 = df::add(df::add(df::mul(dx, dx), df::mul(dy, dy)), df::add(df::mul(dz, dz), df::from_double(eps2)));
    const dfloat ri = df::rsqrt(r2);
    const dfloat w = df::mul(df::mul(df::mul(ri, ri), ri), df::from_double(mj));
    D3 r;
    r.x = df::to_double(df::mul(w, dx));
    r.y = df::to_double(df::mul(w, dy));
    r.z = df::to_double(df::mul(w, dz));
    if (!(isfinite(r.x) && isfinite(r.y) && isfinite(r.z)))
        r = acc_term_fp64(J0, J1, ixh, iyh, izh, ixl, iyl, izl, mj, eps2);
    return r;
}

// A pair term in double-float, and sums of such terms.  The per-thread slot loops add the
// deferred terms of a particle in double-float and convert once: FP64 issues at 1/64 of the
// FP32 rate on this part, and a double per term (its conversions and additions) cost as much
// as the double-float arithmetic itself.
struct DF3 {
    df::dfloat x, y, z;
};

__device__ __forceinline__ DF3 df3_zero()
{
    DF3 r;
    r.x.h = r.x.l = r.y.h = r.y.l = r.z.h = r.z.l = 0.f;
    return r;
}

__device__ __forceinline__ void df3_add(DF3 &a, const DF3 &t)
{
    a.x = df::add(a.x, t.x);
    a.y = df::add(a.y, t.y);
    a.z = df::add(a.z, t.z);
}

__device__ __forceinline__ bool df3_finite(const DF3 &t)
{
    return isfinite(t.x.h) && isfinite(t.y.h) && isfinite(t.z.h) && isfinite(t.x.l) && isfinite(t.y.l) &&
           isfinite(t.z.l);
}

// acc_term_df on position records that carry the double-float mass ({J0.w, J1.w}, the split
// of the FP64 mass that from_double makes) and with the softening as a double-float: no FP64
// instruction.  Returns false when the term leaves the FP32 range (the caller then takes
// acc_term_fp64).
static __device__ __noinline__ bool acc_term_df3(const float4 J0, const float4 J1, float ixh, float iyh, float izh,
                                                 float ixl, float iyl, float izl, df::dfloat e2, DF3 &t)
{
    using df::dfloat;
    const dfloat dx = df::sub(df::make(J0.x, J1.x), df::make(ixh, ixl));
    const dfloat dy = df::sub(df::make(J0.y, J1.y), df::make(iyh, iyl));
    const dfloat dz = df::sub(df::make(J0.z, J1.z), df::make(izh, izl));
    const dfloat r2 = df::add(df::add(df::mul(dx, dx), df::mul(dy, dy)), df::add(df::mul(dz, dz), e2));
    const dfloat ri = df::rsqrt(r2);
    dfloat mj;
    mj.h = J0.w;
    mj.l = J1.w;
    const dfloat w = df::mul(df::mul(df::mul(ri, ri), ri), mj);
    t.x = df::mul(w, dx);
    t.y = df::mul(w, dy);
    t.z = df::mul(w, dz);
    return df3_finite(t);
}

template <int ILP>
struct AccMixedI {
    float xh[ILP], yh[ILP], zh[ILP], xl[ILP], yl[ILP], zl[ILP];
};

// NEWTON: one Newton-Raphson step on the MUFU rsqrt (y <- y (3/2 - r2 y^2 / 2)), for the
// pass that feeds a gradient (the gradient differences a_j - a_i and needs a_j to ~1e-7)
template <int ILP, bool MASK, bool WMAX, bool NEWTON = false>
__device__ __forceinline__ void acc_mixed_j(const float4 J0, const float4 J1, const AccMixedI<ILP> &I,
                                            float eps2, int jpos, const int (&ipos)[ILP],
                                            float (&ax)[ILP], float (&ay)[ILP], float (&az)[ILP],
                                            float (&wm)[ILP])
{
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float dx = (J0.x - I.xh[k]) + (J1.x - I.xl[k]);
        const float dy = (J0.y - I.yh[k]) + (J1.y - I.yl[k]);
        const float dz = (J0.z - I.zh[k]) + (J1.z - I.zl[k]);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        float ri = rsqrtf(r2);
        if (NEWTON) {
            const float hy = (0.5f * r2) * ri;
            ri = fmaf(ri, fmaf(-hy, ri, 0.5f), ri);
        }
        const float ri2 = ri * ri;
        float w = J0.w * ri * ri2;
        if (MASK) w = (jpos == ipos[k]) ? 0.f : w;
        if (WMAX) wm[k] = fmaxf(wm[k], w);
        ax[k] = fmaf(w, dx, ax[k]);
        ay[k] = fmaf(w, dy, ay[k]);
        az[k] = fmaf(w, dz, az[k]);
    }
}

// Newtonian pair term of the pass that feeds a gradient: Newton-refined rsqrt; a term above
// thr[k] goes to a deferred slot and stays out of the FP32 partial sums
template <int ILP, bool MASK, class Slots>
__device__ __forceinline__ void acc_defer_j(const float4 J0, const float4 J1, const AccMixedI<ILP> &I,
                                            float eps2, int jglob, int jpos, const int (&ipos)[ILP],
                                            const float (&thr)[ILP], Slots &big,
                                            float (&ax)[ILP], float (&ay)[ILP], float (&az)[ILP])
{
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float dx = (J0.x - I.xh[k]) + (J1.x - I.xl[k]);
        const float dy = (J0.y - I.yh[k]) + (J1.y - I.yl[k]);
        const float dz = (J0.z - I.zh[k]) + (J1.z - I.zl[k]);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        float ri = rsqrtf(r2);
        const float hy = (0.5f * r2) * ri;
        ri = fmaf(ri, fmaf(-hy, ri, 0.5f), ri);
        float w = J0.w * ri * (ri * ri);
        if (MASK) w = (jpos == ipos[k]) ? 0.f : w;
        const bool isbig = (w > thr[k]) && big.room(k);
        if (isbig) big.push(k, jglob);
        const float wf = isbig ? 0.f : w;
        ax[k] = fmaf(wf, dx, ax[k]);
        ay[k] = fmaf(wf, dy, ay[k]);
        az[k] = fmaf(wf, dz, az[k]);
    }
}

// The scale of the dominant terms, max_j m_j / r^3 = (min_j r^2 m_j^(-2/3))^(-3/2): J1.w holds
// m_j^(-2/3) (set when the tile is staged), so a pair costs the separation, r^2, one product
// and a minimum (no rsqrt); qm[k] is the running minimum of r^2 m_j^(-2/3)
template <int ILP, bool MASK>
__device__ __forceinline__ void wmax_mixed_j(const float4 J0, const float4 J1, const AccMixedI<ILP> &I,
                                             float eps2, int jpos, const int (&ipos)[ILP], float (&qm)[ILP])
{
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float dx = (J0.x - I.xh[k]) + (J1.x - I.xl[k]);
        const float dy = (J0.y - I.yh[k]) + (J1.y - I.yl[k]);
        const float dz = (J0.z - I.zh[k]) + (J1.z - I.zl[k]);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        float q = r2 * J1.w;
        if (MASK) q = (jpos == ipos[k]) ? INFINITY : q;
        qm[k] = fminf(qm[k], q);
    }
}

template <bool MASK>
__device__ __forceinline__ void acc_fp64_j(const double4_32a J, const double4_32a I, double eps2, int jpos,
                                           int ipos, double &ax, double &ay, double &az)
{
    const double dx = J.x - I.x, dy = J.y - I.y, dz = J.z - I.z;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double ri = rsqrt(r2);
    double w = J.w * ri * ri * ri;
    if (MASK) w = (jpos == ipos) ? 0.0 : w;
    ax = fma(w, dx, ax);
    ay = fma(w, dy, ay);
    az = fma(w, dz, az);
}

template <int ILP>
struct GradMixedI {
    float xh[ILP], yh[ILP], zh[ILP], xm[ILP], ym[ILP], zm[ILP], xl[ILP], yl[ILP], zl[ILP];
    float ahx[ILP], ahy[ILP], ahz[ILP], alx[ILP], aly[ILP], alz[ILP];
};

// The gradient pair term of grad_term_df in FP64 from the same split records (their parts
// sum exactly in FP64), for a pair whose double-float evaluation leaves the FP32 exponent
// range: near the pericentre of a hard binary m r^-5 |a_ji| r^2 reaches ~1e41 (r ~ 1e-10 in
// Henon units), above the largest FP32 value, 3.4e38.
template <int ILP>
__device__ __noinline__ void grad_term_fp64(const float4 J0, const float4 J1, const float4 J2, const float4 J3,
                                            const GradMixedI<ILP> &I, int k, double eps2, double &gx, double &gy,
                                            double &gz)
{
    const double dx = ((double)J0.x + (double)J1.x + (double)J2.x) - ((double)I.xh[k] + (double)I.xm[k] + (double)I.xl[k]);
    const double dy = ((double)J0.y + (double)J1.y + (double)J2.y) - ((double)I.yh[k] + (double)I.ym[k] + (double)I.yl[k]);
    const double dz = ((double)J0.z + (double)J1.z + (double)J2.z) - ((double)I.zh[k] + (double)I.zm[k] + (double)I.zl[k]);
    const double Ax = ((double)J1.w + (double)J3.y) - ((double)I.ahx[k] + (double)I.alx[k]);
    const double Ay = ((double)J2.w + (double)J3.z) - ((double)I.ahy[k] + (double)I.aly[k]);
    const double Az = ((double)J3.x + (double)J3.w) - ((double)I.ahz[k] + (double)I.alz[k]);
    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
    const double ri = 1.0 / sqrt(r2);
    const double ri2 = ri * ri;
    const double w = (double)J0.w * ri2 * ri;
    const double t3 = 3.0 * (dx * Ax + dy * Ay + dz * Az) * ri2;
    gx += w * (Ax - t3 * dx);
    gy += w * (Ay - t3 * dy);
    gz += w * (Az - t3 * dz);
}

// One gradient pair term in double-float, rebuilt from the split records (positions to 48
// bits, accelerations to 36 bits); used for the few dominant terms of each particle.  A term
// outside the FP32 exponent range is evaluated in FP64 instead (grad_term_fp64).
template <int ILP>
__device__ __noinline__ void grad_term_df(const float4 J0, const float4 J1, const float4 J2, const float4 J3,
                                          const GradMixedI<ILP> &I, int k, double eps2, double &gx, double &gy,
                                          double &gz)
{
    using df::dfloat;
    const dfloat dx = df::sep(J0.x, J1.x, J2.x, I.xh[k], I.xm[k], I.xl[k]);
    const dfloat dy = df::sep(J0.y, J1.y, J2.y, I.yh[k], I.ym[k], I.yl[k]);
    const dfloat dz = df::sep(J0.z, J1.z, J2.z, I.zh[k], I.zm[k], I.zl[k]);
    const dfloat Ax = df::sub(df::make(J1.w, J3.y), df::make(I.ahx[k], I.alx[k]));
    const dfloat Ay = df::sub(df::make(J2.w, J3.z), df::make(I.ahy[k], I.aly[k]));
    const dfloat Az = df::sub(df::make(J3.x, J3.w), df::make(I.ahz[k], I.alz[k]));
    const dfloat r2 = df::add(df::add(df::mul(dx, dx), df::mul(dy, dy)), df::add(df::mul(dz, dz), df::from_double(eps2)));
    const dfloat ri = df::rsqrt(r2);
    const dfloat ri2 = df::mul(ri, ri);
    const dfloat w = df::mul_f(df::mul(ri2, ri), J0.w);
    const dfloat xa = df::add(df::add(df::mul(dx, Ax), df::mul(dy, Ay)), df::mul(dz, Az));
    const dfloat t3 = df::mul(df::mul_f(xa, 3.f), ri2);
    const double tx = df::to_double(df::mul(w, df::sub(Ax, df::mul(t3, dx))));
    const double ty = df::to_double(df::mul(w, df::sub(Ay, df::mul(t3, dy))));
    const double tz = df::to_double(df::mul(w, df::sub(Az, df::mul(t3, dz))));
    if (isfinite(tx) && isfinite(ty) && isfinite(tz)) {
        gx += tx;
        gy += ty;
        gz += tz;
    } else {
        grad_term_fp64<ILP>(J0, J1, J2, J3, I, k, eps2, gx, gy, gz);
    }
}

// grad_term_df with the softening as a double-float and the result as one (no FP64
// instruction); false when the term leaves the FP32 range (the caller takes grad_term_fp64)
template <int ILP>
__device__ __noinline__ bool grad_term_df3(const float4 J0, const float4 J1, const float4 J2, const float4 J3,
                                           const GradMixedI<ILP> &I, int k, df::dfloat e2, DF3 &t)
{
    using df::dfloat;
    const dfloat dx = df::sep(J0.x, J1.x, J2.x, I.xh[k], I.xm[k], I.xl[k]);
    const dfloat dy = df::sep(J0.y, J1.y, J2.y, I.yh[k], I.ym[k], I.yl[k]);
    const dfloat dz = df::sep(J0.z, J1.z, J2.z, I.zh[k], I.zm[k], I.zl[k]);
    const dfloat Ax = df::sub(df::make(J1.w, J3.y), df::make(I.ahx[k], I.alx[k]));
    const dfloat Ay = df::sub(df::make(J2.w, J3.z), df::make(I.ahy[k], I.aly[k]));
    const dfloat Az = df::sub(df::make(J3.x, J3.w), df::make(I.ahz[k], I.alz[k]));
    const dfloat r2 = df::add(df::add(df::mul(dx, dx), df::mul(dy, dy)), df::add(df::mul(dz, dz), e2));
    const dfloat ri = df::rsqrt(r2);
    const dfloat ri2 = df::mul(ri, ri);
    const dfloat w = df::mul_f(df::mul(ri2, ri), J0.w);
    const dfloat xa = df::add(df::add(df::mul(dx, Ax), df::mul(dy, Ay)), df::mul(dz, Az));
    const dfloat t3 = df::mul(df::mul_f(xa, 3.f), ri2);
    t.x = df::mul(w, df::sub(Ax, df::mul(t3, dx)));
    t.y = df::mul(w, df::sub(Ay, df::mul(t3, dy)));
    t.z = df::mul(w, df::sub(Az, df::mul(t3, dz)));
    return df3_finite(t);
}

template <int ILP, bool MASK, class Slots>
__device__ __forceinline__ void grad_mixed_j(const float4 J0, const float4 J1, const float4 J2,
                                             const float4 J3, const GradMixedI<ILP> &I,
                                             float eps2, int jglob, int jpos,
                                             const int (&ipos)[ILP], const float (&thr)[ILP],
                                             Slots &big, float (&gx)[ILP],
                                             float (&gy)[ILP], float (&gz)[ILP])
{
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        // separation: the high and middle parts subtract exactly, one rounding at the end
        const float dx = ((J0.x - I.xh[k]) + (J1.x - I.xm[k])) + (J2.x - I.xl[k]);
        const float dy = ((J0.y - I.yh[k]) + (J1.y - I.ym[k])) + (J2.y - I.yl[k]);
        const float dz = ((J0.z - I.zh[k]) + (J1.z - I.zm[k])) + (J2.z - I.zl[k]);
        // a_ji = a_j - a_i from the 12-bit split (exact high-part difference)
        const float Ax = (J1.w - I.ahx[k]) + (J3.y - I.alx[k]);
        const float Ay = (J2.w - I.ahy[k]) + (J3.z - I.aly[k]);
        const float Az = (J3.x - I.ahz[k]) + (J3.w - I.alz[k]);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        float y = rsqrtf(r2);
        // one Newton-Raphson step for 1/sqrt(r2): y <- y (3/2 - r2 y^2 / 2)
        const float hy = (0.5f * r2) * y;
        y = fmaf(y, fmaf(-hy, y, 0.5f), y);
        const float ri2 = y * y;
        float w = J0.w * y * ri2;  // m_j r^-3
        bool self = false;
        if (MASK) {
            self = (jpos == ipos[k]);
            w = self ? 0.f : w;
        }
        // a dominant term goes to a deferred double-float slot and stays out of the FP32 sum
        const bool isbig = (w > thr[k]) && big.room(k);
        if (isbig) big.push(k, jglob);
        const float wf = isbig ? 0.f : w;
        const float xa = fmaf(dx, Ax, fmaf(dy, Ay, dz * Az));
        const float t3 = 3.0f * xa * ri2;  // 3 (x.a) / r^2
        const float nx = fmaf(wf, fmaf(-t3, dx, Ax), gx[k]);
        const float ny = fmaf(wf, fmaf(-t3, dy, Ay), gy[k]);
        const float nz = fmaf(wf, fmaf(-t3, dz, Az), gz[k]);
        if (MASK) {
            gx[k] = self ? gx[k] : nx;
            gy[k] = self ? gy[k] : ny;
            gz[k] = self ? gz[k] : nz;
        } else {
            gx[k] = nx;
            gy[k] = ny;
            gz[k] = nz;
        }
    }
}

// The thread's two particles as the two lanes of packed f32x2 arithmetic (negated parts)
struct GradX2I {
    float2 nxh, nyh, nzh, nxm, nym, nzm, nxl, nyl, nzl, nahx, nahy, nahz, nalx, naly, nalz;
};

// One source, staged duplicated as G0 {xh, xh, yh, yh}, G1 {zh, zh, xm, xm}, G2 {ym, ym, zm, zm},
// G3 {xl, xl, yl, yl}, G4 {zl, zl, ahx, ahx}, G5 {ahy, ahy, ahz, ahz}, G6 {alx, alx, aly, aly},
// G7 {alz, alz, m, m}, against the thread's two particles.  The operations and their order
// are those of grad_mixed_j, lane by lane.
template <class Slots>
__device__ __forceinline__ void grad_x2_j(const float4 G0, const float4 G1, const float4 G2, const float4 G3,
                                          const float4 G4, const float4 G5, const float4 G6, const float4 G7,
                                          const GradX2I &P, float2 e2, int jglob, const float (&thr)[2],
                                          Slots &big, float2 &gx, float2 &gy, float2 &gz)
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
    float2 w = __fmul2_rn(__fmul2_rn(make_float2(G7.z, G7.w), y), ri2);  // m_j r^-3
    // a dominant term goes to a deferred double-float slot and stays out of the FP32 sum
    // (a warp vote before this, as in acc_x2_j, costs two registers here and a block per SM)
    const bool b0 = (w.x > thr[0]) && big.room(0);
    if (b0) big.push(0, jglob);
    const bool b1 = (w.y > thr[1]) && big.room(1);
    if (b1) big.push(1, jglob);
    w.x = b0 ? 0.f : w.x;
    w.y = b1 ? 0.f : w.y;
    const float2 xa = __ffma2_rn(dx, Ax, __ffma2_rn(dy, Ay, __fmul2_rn(dz, Az)));
    const float2 nt3 = __fmul2_rn(__fmul2_rn(make_float2(-3.0f, -3.0f), xa), ri2);  // -3 (x.a) / r^2
    gx = __ffma2_rn(w, __ffma2_rn(nt3, dx, Ax), gx);
    gy = __ffma2_rn(w, __ffma2_rn(nt3, dy, Ay), gy);
    gz = __ffma2_rn(w, __ffma2_rn(nt3, dz, Az), gz);
}

template <bool MASK>
__device__ __forceinline__ void grad_fp64_j(const double4_32a J, const double4_32a JA, const double4_32a I,
                                            const double4_32a IA, double eps2, int jpos, int ipos,
                                            double &gx, double &gy, double &gz)
{
    const double dx = J.x - I.x, dy = J.y - I.y, dz = J.z - I.z;
    const double Ax = JA.x - IA.x, Ay = JA.y - IA.y, Az = JA.z - IA.z;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double ri = rsqrt(r2);
    const double ri2 = ri * ri;
    const double w = J.w * ri * ri2;
    const double xa = fma(dx, Ax, fma(dy, Ay, dz * Az));
    const double t3 = 3.0 * xa * ri2;
    const double nx = fma(w, fma(-t3, dx, Ax), gx);
    const double ny = fma(w, fma(-t3, dy, Ay), gy);
    const double nz = fma(w, fma(-t3, dz, Az), gz);
    if (MASK && jpos == ipos) return;
    gx = nx;
    gy = ny;
    gz = nz;
}

// symmetrisation factor s(d) = tau_sym / tau (Eq. time-step-factor)
template <int SYM>
__device__ __forceinline__ float symf(float d)
{
    if (SYM == 0) {
        // harmonic: with q = 1 + sqrt(1 + d^2) the printed factor equals (q + d) / q and
        // 2 / (q - d); each form is used where it has no cancellation
        const float q = 1.f + sqrtf(fmaf(d, d, 1.f));
        const float num = (d >= 0.f) ? q + d : 2.f;
        const float den = (d >= 0.f) ? q : q - d;
        return __fdividef(num, den);
    } else if (SYM == 1) {
        // arithmetic: 1 / (1 - d/2) for d < 2; beyond, the step is lowered by 1/d first
        return (d < 2.f) ? __fdividef(1.f, fmaf(-0.5f, d, 1.f)) : __fdividef(2.f, d);
    } else {
        return 1.f;
    }
}

template <int SYM>
__device__ __forceinline__ double symd(double d)
{
    if (SYM == 0) {
        const double q = 1.0 + sqrt(fma(d, d, 1.0));
        return (d >= 0.0) ? (q + d) / q : 2.0 / (q - d);
    } else if (SYM == 1) {
        return (d < 2.0) ? 1.0 / (1.0 - 0.5 * d) : 2.0 / d;
    } else {
        return 1.0;
    }
}

template <int ILP>
struct TstepMixedI {
    float xh[ILP], yh[ILP], zh[ILP], xl[ILP], yl[ILP], zl[ILP], vx[ILP], vy[ILP], vz[ILP], gm[ILP];
    float ax[ILP], ay[ILP], az[ILP];  // used with the exact fly-by derivative (SYM & 4)
};

// Pair time-steps without eta: best[k] = min(best[k], tau_ff_sym, tau_fb_sym), minr2[k] =
// min(minr2[k], r^2).  Every symmetrisation factor obeys s(d) >= 1 / (1 + |d|) (harmonic:
// q - d <= 2 (1 + |d|); arithmetic: 1 / (1 + |d|/2) and 2 / d; none: 1), so a criterion with
// t >= bnd (1 + |d|), bnd = 1.001 best, cannot lower the minimum; it is not symmetrised, and
// the warp skips the factors (two MUFU sqrt/divide pairs) when no lane needs them.  The 0.1%
// margin is far above the rounding of the test and of the factor, so the result is the one
// of the full evaluation.  Each d is t times a rate (dt/dt / t), so the test is written
// t - |bnd d / t| t >= bnd: one FMA per criterion with the rate scaled by bnd eta, and d
// itself is formed only for the pairs that pass.  An unordered test (a NaN, e.g. from
// bnd = inf before the first pair) counts as "may lower": such a pair is evaluated, and a
// NaN result leaves best unchanged under fminf.
// SYM & 3 selects the factor (0 harmonic, 1 arithmetic, 2 none); SYM & 4 the exact fly-by
// derivative [r.v/r^2 - v.a/v^2] t_fb with the relative acceleration JA - I.a (first line of
// Eq. dt-flyby-derivative) instead of its two-body approximation.
template <int ILP, int SYM, bool MASK>
__device__ __forceinline__ void tstep_mixed_j(const float4 J0, const float4 J1, const float4 JV, const float4 JA,
                                              const TstepMixedI<ILP> &I, float eta, float eta15,
                                              int jpos, const int (&ipos)[ILP],
                                              float (&best)[ILP], float (&minr2)[ILP])
{
    float tff[ILP], tfb[ILP], rvr2[ILP], hfb[ILP];
    bool nff[ILP], nfb[ILP];
    bool any = false;
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float dx = (J0.x - I.xh[k]) + (J1.x - I.xl[k]);
        const float dy = (J0.y - I.yh[k]) + (J1.y - I.yl[k]);
        const float dz = (J0.z - I.zh[k]) + (J1.z - I.zl[k]);
        const float ux = JV.x - I.vx[k], uy = JV.y - I.vy[k], uz = JV.z - I.vz[k];
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float v2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float rv = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
        const float ri = rsqrtf(r2);
        const float ri2 = ri * ri;
        const float gm = I.gm[k] + JV.w;            // G (m_i + m_j)
        tff[k] = rsqrtf(gm * ri2 * ri);              // (r^3 / (G M))^(1/2)
        rvr2[k] = rv * ri2;                          // r.v / r^2
        const float iv = rsqrtf(v2);                 // 1 / |v|
        tfb[k] = r2 * ri * iv;                       // r / |v|
        const float bnd = 1.001f * best[k];
        const float ce = bnd * eta;
        const float z = ce * rvr2[k];                // bnd dt_ff/dt / (1.5 t_ff)
        float mfb;
        if (SYM & 4) {
            const float wx = JA.x - I.ax[k], wy = JA.y - I.ay[k], wz = JA.z - I.az[k];
            const float va = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
            hfb[k] = fmaf(-va, iv * iv, rvr2[k]);    // dt_fb/dt / t_fb, exact
            mfb = -fabsf(ce * hfb[k]);
        } else {
            hfb[k] = fmaf(gm * ri, iv * iv, 1.f);    // dt_fb/dt / (t_fb r.v/r^2), two-body
            mfb = -fabsf(z) * hfb[k];
        }
        float rr = r2;
        bool self = false;
        if (MASK) {
            self = (jpos == ipos[k]);
            rr = self ? INFINITY : rr;
        }
        minr2[k] = fminf(minr2[k], rr);
        nff[k] = !self && !(fmaf(-1.5f * fabsf(z), tff[k], tff[k]) >= bnd);
        nfb[k] = !self && (v2 > 0.f) && !(fmaf(mfb, tfb[k], tfb[k]) >= bnd);
        any = any || nff[k] || nfb[k];
    }
    if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            float t = INFINITY;
            if (nff[k]) t = tff[k] * symf<(SYM & 3)>(eta15 * rvr2[k] * tff[k]);
            if (nfb[k]) {
                const float dfb = (SYM & 4) ? eta * hfb[k] * tfb[k] : eta * rvr2[k] * hfb[k] * tfb[k];
                t = fminf(t, tfb[k] * symf<(SYM & 3)>(dfb));
            }
            best[k] = fminf(best[k], t);
        }
    }
}

// The thread's two particles as the two lanes of packed f32x2 arithmetic (negated parts)
struct TstepX2I {
    float2 nxh, nyh, nzh, nxl, nyl, nzl, nvx, nvy, nvz, gm, nax, nay, naz;
};

// One source, staged duplicated as A {hx, hx, hy, hy}, B {hz, hz, lx, lx}, C {ly, ly, lz, lz},
// V0 {vx, vx, vy, vy}, V1 {vz, vz, Gm, Gm} and, with the exact fly-by derivative, W0 {ax, ax,
// ay, ay}, W1 {az, az, 0, 0}, against the thread's two particles.  The operations and their
// order are those of tstep_mixed_j, lane by lane; bnd = 1.001 best and ce = bnd eta are kept
// by the caller (initially inf) and renewed here when best changes.
template <int SYM>
__device__ __forceinline__ void tstep_x2_j(const float4 A, const float4 B, const float4 C, const float4 V0,
                                           const float4 V1, const float4 W0, const float4 W1, const TstepX2I &P,
                                           float eta, float eta15, float (&best)[2], float (&minr2)[2],
                                           float (&bnd)[2], float (&ce)[2])
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
    const float2 gm = __fadd2_rn(P.gm, make_float2(V1.z, V1.w));  // G (m_i + m_j)
    const float2 q = __fmul2_rn(__fmul2_rn(gm, ri2), ri);
    const float2 tff = make_float2(rsqrtf(q.x), rsqrtf(q.y));  // (r^3 / (G M))^(1/2)
    const float2 rvr2 = __fmul2_rn(rv, ri2);                    // r.v / r^2
    const float2 iv = make_float2(rsqrtf(v2.x), rsqrtf(v2.y));  // 1 / |v|
    const float2 tfb = __fmul2_rn(__fmul2_rn(r2, ri), iv);      // r / |v|
    const float2 z = __fmul2_rn(make_float2(ce[0], ce[1]), rvr2);
    float2 hfb, mfb;
    if (SYM & 4) {
        const float2 wx = __fadd2_rn(make_float2(W0.x, W0.y), P.nax);
        const float2 wy = __fadd2_rn(make_float2(W0.z, W0.w), P.nay);
        const float2 wz = __fadd2_rn(make_float2(W1.x, W1.y), P.naz);
        const float2 va = __ffma2_rn(ux, wx, __ffma2_rn(uy, wy, __fmul2_rn(uz, wz)));
        // fma(-va, iv^2, rvr2) as fma(va, -(iv^2), rvr2)
        const float2 niv2 = __fmul2_rn(__fmul2_rn(make_float2(-1.f, -1.f), iv), iv);
        hfb = __ffma2_rn(va, niv2, rvr2);
        const float2 zb = __fmul2_rn(make_float2(ce[0], ce[1]), hfb);
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
        minr2[k] = fminf(minr2[k], rr[k]);
        nff[k] = !(lf[k] >= bnd[k]);
        nfb[k] = (vv[k] > 0.f) && !(lb[k] >= bnd[k]);
        any = any || nff[k] || nfb[k];
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
            best[k] = fminf(best[k], t);
            bnd[k] = 1.001f * best[k];
            ce[k] = bnd[k] * eta;
        }
    }
}

// FP64 pair time-steps, with the same bound on the symmetrisation factors
template <int SYM, bool MASK>
__device__ __forceinline__ void tstep_fp64_j(const double4_32a J, const double4_32a JV, const double4_32a JA,
                                             const double4_32a I, const double4_32a IV, const double4_32a IA,
                                             double eta, int jpos, int ipos, double &best, double &minr2)
{
    const double dx = J.x - I.x, dy = J.y - I.y, dz = J.z - I.z;
    const double ux = JV.x - IV.x, uy = JV.y - IV.y, uz = JV.z - IV.z;
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double v2 = fma(ux, ux, fma(uy, uy, uz * uz));
    const double rv = fma(dx, ux, fma(dy, uy, dz * uz));
    const double r = sqrt(r2);
    const double gm = IV.w + JV.w;
    const double tff = sqrt(r2 * r / gm);
    const double rvr2 = rv / r2;
    const double dff = eta * 1.5 * rvr2 * tff;
    double tfb = INFINITY, dfb = 0.0;
    if (v2 > 0.0) {
        tfb = r / sqrt(v2);
        if (SYM & 4) {
            const double va = fma(ux, JA.x - IA.x, fma(uy, JA.y - IA.y, uz * (JA.z - IA.z)));
            dfb = eta * (rvr2 - va / v2) * tfb;
        } else {
            dfb = eta * rvr2 * (1.0 + gm / (v2 * r)) * tfb;
        }
    }
    const bool self = MASK && jpos == ipos;
    if (!self) minr2 = fmin(minr2, r2);
    const double bnd = 1.001 * best;
    const bool nff = !self && (tff < bnd * (1.0 + fabs(dff)));
    const bool nfb = !self && (v2 > 0.0) && (tfb < bnd * (1.0 + fabs(dfb)));
    if (__any_sync(0xffffffffu, nff || nfb)) {
        double t = INFINITY;
        if (nff) t = tff * symd<(SYM & 3)>(dff);
        if (nfb) t = fmin(t, tfb * symd<(SYM & 3)>(dfb));
        best = fmin(best, t);
    }
}


// ======================================================================================
// Per-i-block bodies.  Each processes the active records [ibase, ibase + BS*ILP) against the
// source records [jb, je), staging the sources through shared memory in tiles of TJ, and
// leaves per-thread results in registers.  Every thread of the block must call a body (it
// synchronises the block); thread t owns the active particles ibase + k*BS + t, k < ILP.
// The grid kernels call a body once per (i-block, j-split) block; the single-CTA subtree
// solver calls it for every i-block of a set against the whole source list.
// ======================================================================================

// The thread's two particles as the two lanes of packed f32x2 arithmetic (negated positions,
// so that a separation is two packed adds: x_j + (-x_i))
struct AccX2I {
    float2 nxh, nyh, nzh, nxl, nyl, nzl;
};

// One source (staged duplicated: A = {hx, hx, hy, hy}, B = {hz, hz, lx, lx},
// C = {ly, ly, lz, lz}, M = {m, m}) against the thread's two particles.  The operations and
// their order are those of acc_mixed_j (and acc_defer_j when DEFER), lane by lane, so the
// packed and scalar loops give the same bits.
template <bool WMAX, bool NEWTON, bool DEFER, class Slots>
__device__ __forceinline__ void acc_x2_j(const float4 A, const float4 B, const float4 C, const float2 M,
                                         const AccX2I &P, float2 e2, int jglob, const float (&thr)[2],
                                         Slots &big, float2 &ax, float2 &ay, float2 &az, float (&wm)[2])
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), P.nxh), __fadd2_rn(make_float2(B.z, B.w), P.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), P.nyh), __fadd2_rn(make_float2(C.x, C.y), P.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), P.nzh), __fadd2_rn(make_float2(C.z, C.w), P.nzl));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (NEWTON) {
        // y <- y (3/2 - r2 y^2 / 2) as fma(y, fma(-(r2/2) y, y, 1/2), y)
        const float2 nhy = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), r2), ri);
        ri = __ffma2_rn(ri, __ffma2_rn(nhy, ri, make_float2(0.5f, 0.5f)), ri);
    }
    float2 w = __fmul2_rn(__fmul2_rn(M, ri), __fmul2_rn(ri, ri));
    if (WMAX) {
        wm[0] = fmaxf(wm[0], w.x);
        wm[1] = fmaxf(wm[1], w.y);
    }
    if (DEFER) {
        // most warp-steps have no candidate at all: one vote skips the per-lane slot logic
        if (__any_sync(0xffffffffu, (w.x > thr[0]) || (w.y > thr[1]))) {
            const bool b0 = (w.x > thr[0]) && big.room(0);
            if (b0) big.push(0, jglob);
            const bool b1 = (w.y > thr[1]) && big.room(1);
            if (b1) big.push(1, jglob);
            w.x = b0 ? 0.f : w.x;
            w.y = b1 ? 0.f : w.y;
        }
    }
    ax = __ffma2_rn(w, dx, ax);
    ay = __ffma2_rn(w, dy, ay);
    az = __ffma2_rn(w, dz, az);
}

// Newtonian pass, mixed precision (float-float separations, MUFU rsqrt, folds every 64)
// NEWTON (the pass that feeds a gradient): Newton-refined rsqrt and folds every 16 pairs.
// DEFER (with NEWTON): the terms above SLOT_FRACTION x wmax[i] (wmax from a prepass at the
// same positions) are deferred and summed in double-float after the loop, with the FP64
// masses mstore[jlist[j]] (jlist NULL: the identity).
template <int BS, int ILP, int TJ, bool WMAX, bool NEWTON = false, bool DEFER = false>
__device__ __forceinline__ void acc_mixed_body(const float4 *__restrict__ irec,
                                               const float4 *__restrict__ jrec, int n_a, int n_s,
                                               int ibase, int jb, int je, int self_pass, float eps2,
                                               double (&res)[ILP][3], float (&wres)[ILP],
                                               const float *__restrict__ wmax = nullptr, double eps2d = 0.0,
                                               const int32_t *__restrict__ jlist = nullptr,
                                               const double *__restrict__ mstore = nullptr)
{
    static_assert(!DEFER || NEWTON, "the deferred variant is the accurate one");
    // ILP == 2: sources staged duplicated for the packed loop; otherwise as {hi, m}, {lo, 0}
    constexpr bool X2 = (ILP == 2);
    __shared__ float4 s0[X2 ? 1 : TJ];
    __shared__ float4 s1[X2 ? 1 : TJ];
    __shared__ float4 sA[X2 ? TJ : 1], sB[X2 ? TJ : 1], sC[X2 ? TJ : 1];
    __shared__ float2 sM[X2 ? TJ : 1];
    const int tid = threadIdx.x;
    AccMixedI<ILP> I;
    int ipos[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + tid;
        ipos[k] = i;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (i < n_a) {
            a = irec[i];
            b = irec[n_a + i];
        }
        I.xh[k] = a.x; I.yh[k] = a.y; I.zh[k] = a.z;
        I.xl[k] = b.x; I.yl[k] = b.y; I.zl[k] = b.z;
    }
    float thr[ILP];
    SmemSlots<ILP, BS> big;
    if constexpr (DEFER) {
        __shared__ int s_slot[GRAD_SLOTS * ILP * BS];
        big.col = s_slot + tid;
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            big.n[k] = 0;
            thr[k] = (ipos[k] < n_a) ? SLOT_FRACTION * wmax[ipos[k]] : INFINITY;
        }
    }
    float hx[ILP], hy[ILP], hz[ILP], lx[ILP], ly[ILP], lz[ILP], wm[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = wm[k] = 0.f;

    // FP32 partial sums over at most FOLD pairs before each compensated fold
    constexpr int FOLD = NEWTON ? 16 : 64;
    if constexpr (X2) {
        AccX2I P;
        P.nxh = make_float2(-I.xh[0], -I.xh[1]);
        P.nyh = make_float2(-I.yh[0], -I.yh[1]);
        P.nzh = make_float2(-I.zh[0], -I.zh[1]);
        P.nxl = make_float2(-I.xl[0], -I.xl[1]);
        P.nyl = make_float2(-I.yl[0], -I.yl[1]);
        P.nzl = make_float2(-I.zl[0], -I.zl[1]);
        const float2 e2 = make_float2(eps2, eps2);
        const float (&thr2)[2] = *reinterpret_cast<const float(*)[2]>(thr);
        float (&wm2)[2] = *reinterpret_cast<float(*)[2]>(wm);
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
                const float4 a = jrec[j0 + t];
                const float4 b = jrec[n_s + j0 + t];
                sA[t] = make_float4(a.x, a.x, a.y, a.y);
                sB[t] = make_float4(a.z, a.z, b.x, b.x);
                sC[t] = make_float4(b.y, b.y, b.z, b.z);
                sM[t] = make_float2(a.w, a.w);
            }
            __syncthreads();
            const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
            for (int c0 = 0; c0 < cnt; c0 += FOLD) {
                const int c1 = min(cnt, c0 + FOLD);
                float2 ax2 = make_float2(0.f, 0.f), ay2 = ax2, az2 = ax2;
                if (!diag) {
                    int jj = c0;
                    for (; jj + 8 <= c1; jj += 8) {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            acc_x2_j<WMAX, NEWTON, DEFER>(sA[jj + u], sB[jj + u], sC[jj + u], sM[jj + u], P, e2,
                                                          j0 + jj + u, thr2, big, ax2, ay2, az2, wm2);
                    }
                    for (; jj < c1; ++jj)
                        acc_x2_j<WMAX, NEWTON, DEFER>(sA[jj], sB[jj], sC[jj], sM[jj], P, e2, j0 + jj, thr2, big, ax2,
                                                      ay2, az2, wm2);
                } else {
                    // the i = j term masked by list position: the scalar bodies
                    float ax[ILP] = {0.f, 0.f}, ay[ILP] = {0.f, 0.f}, az[ILP] = {0.f, 0.f};
                    for (int jj = c0; jj < c1; ++jj) {
                        const float4 A = sA[jj], B = sB[jj], C = sC[jj];
                        const float4 J0 = make_float4(A.x, A.z, B.x, sM[jj].x);
                        const float4 J1 = make_float4(B.z, C.x, C.z, 0.f);
                        if constexpr (DEFER)
                            acc_defer_j<ILP, true>(J0, J1, I, eps2, j0 + jj, j0 + jj, ipos, thr, big, ax, ay, az);
                        else
                            acc_mixed_j<ILP, true, WMAX, NEWTON>(J0, J1, I, eps2, j0 + jj, ipos, ax, ay, az, wm);
                    }
                    ax2 = make_float2(ax[0], ax[1]);
                    ay2 = make_float2(ay[0], ay[1]);
                    az2 = make_float2(az[0], az[1]);
                }
                fold2(hx[0], lx[0], ax2.x);
                fold2(hy[0], ly[0], ay2.x);
                fold2(hz[0], lz[0], az2.x);
                fold2(hx[1], lx[1], ax2.y);
                fold2(hy[1], ly[1], ay2.y);
                fold2(hz[1], lz[1], az2.y);
            }
        }
    } else {
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            s0[t] = jrec[j0 + t];
            s1[t] = jrec[n_s + j0 + t];
        }
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
        for (int c0 = 0; c0 < cnt; c0 += FOLD) {
            const int c1 = min(cnt, c0 + FOLD);
            float ax[ILP], ay[ILP], az[ILP];
#pragma unroll
            for (int k = 0; k < ILP; ++k) ax[k] = ay[k] = az[k] = 0.f;
            int jj = c0;
            if constexpr (DEFER) {
                if (!diag) {
                    for (; jj + 8 <= c1; jj += 8) {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            acc_defer_j<ILP, false>(s0[jj + u], s1[jj + u], I, eps2, j0 + jj + u, 0, ipos, thr, big,
                                                    ax, ay, az);
                    }
                    for (; jj < c1; ++jj)
                        acc_defer_j<ILP, false>(s0[jj], s1[jj], I, eps2, j0 + jj, 0, ipos, thr, big, ax, ay, az);
                } else {
                    for (; jj < c1; ++jj)
                        acc_defer_j<ILP, true>(s0[jj], s1[jj], I, eps2, j0 + jj, j0 + jj, ipos, thr, big, ax, ay,
                                               az);
                }
            } else if (!diag) {
                for (; jj + 8 <= c1; jj += 8) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        acc_mixed_j<ILP, false, WMAX, NEWTON>(s0[jj + u], s1[jj + u], I, eps2, 0, ipos, ax, ay, az,
                                                              wm);
                }
                for (; jj < c1; ++jj)
                    acc_mixed_j<ILP, false, WMAX, NEWTON>(s0[jj], s1[jj], I, eps2, 0, ipos, ax, ay, az, wm);
            } else {
                for (; jj < c1; ++jj)
                    acc_mixed_j<ILP, true, WMAX, NEWTON>(s0[jj], s1[jj], I, eps2, j0 + jj, ipos, ax, ay, az, wm);
            }
#pragma unroll
            for (int k = 0; k < ILP; ++k) {
                fold2(hx[k], lx[k], ax[k]);
                fold2(hy[k], ly[k], ay[k]);
                fold2(hz[k], lz[k], az[k]);
            }
        }
    }
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        res[k][0] = (double)hx[k] + (double)lx[k];
        res[k][1] = (double)hy[k] + (double)ly[k];
        res[k][2] = (double)hz[k] + (double)lz[k];
        wres[k] = wm[k];
    }
    if constexpr (DEFER && BS == 32) {
        // deferred double-float terms of the one-warp (small-tile) layout, shared by the lanes;
        // source records read back from global memory (L2), the owner's own record from irec
        __shared__ D3 s_xbuf[BS];
        __syncwarp();
        warp_slot_terms<ILP>(big.n, s_xbuf, res, [&](int ol, int k, int s) -> D3 {
            const int j = big.col[(s * ILP + k) * BS + ol - tid];
            const int i = ibase + k * BS + ol;
            const float4 a = irec[i], b = irec[n_a + i];
            const double mj = mstore[jlist ? jlist[j] : j];
            return acc_term_df(jrec[j], jrec[n_s + j], a.x, a.y, a.z, b.x, b.y, b.z, mj, eps2d);
        });
    } else if constexpr (DEFER) {
        // deferred double-float terms, per thread, summed in double-float; records read back
        // from global memory (L2)
        const df::dfloat e2 = df::from_double(eps2d);
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            DF3 b = df3_zero();
            double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int s = 0; s < GRAD_SLOTS; ++s) {
                if (s < big.n[k]) {
                    const int j = big.get(s, k);
                    const float4 J0 = jrec[j], J1 = jrec[n_s + j];
                    DF3 t;
                    if (acc_term_df3(J0, J1, I.xh[k], I.yh[k], I.zh[k], I.xl[k], I.yl[k], I.zl[k], e2, t)) {
                        df3_add(b, t);
                    } else {
                        const D3 u = acc_term_fp64(J0, J1, I.xh[k], I.yh[k], I.zh[k], I.xl[k], I.yl[k], I.zl[k],
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
    }
}

// max_j m_j / r^3 over [jb, je) for the active records of the block (the prepass of the
// deferred Newtonian pass).  With two particles a thread (ILP = 2) the off-diagonal tiles run
// on packed f32x2 arithmetic: the thread's two particles are the two lanes, and the sources
// are staged duplicated ({x, x}, ...) so that every operand is a register pair as loaded.
// The operations and their order are those of wmax_mixed_j, so the result is bit-identical.
template <int BS, int ILP, int TJ>
__device__ __forceinline__ void wmax_mixed_body(const float4 *__restrict__ irec,
                                                const float4 *__restrict__ jrec, int n_a, int n_s,
                                                int ibase, int jb, int je, int self_pass, float eps2,
                                                float (&wres)[ILP])
{
    // per source: {hx, hx, hy, hy}, {hz, hz, lx, lx}, {ly, ly, lz, lz}, {mq, mq} with
    // mq = m^(-2/3) (infinite for a massless source, which then never sets the minimum)
    __shared__ float4 sA[TJ], sB[TJ], sC[TJ];
    __shared__ float2 sM[TJ];
    const int tid = threadIdx.x;
    AccMixedI<ILP> I;
    int ipos[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + tid;
        ipos[k] = i;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (i < n_a) {
            a = irec[i];
            b = irec[n_a + i];
        }
        I.xh[k] = a.x; I.yh[k] = a.y; I.zh[k] = a.z;
        I.xl[k] = b.x; I.yl[k] = b.y; I.zl[k] = b.z;
        wres[k] = INFINITY;  // the running minimum of r^2 m_j^(-2/3) until the end
    }
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            const float4 a = jrec[j0 + t];
            const float4 b = jrec[n_s + j0 + t];
            const float mq = (a.w > 0.f) ? exp2f(-0.6666667f * log2f(a.w)) : INFINITY;
            sA[t] = make_float4(a.x, a.x, a.y, a.y);
            sB[t] = make_float4(a.z, a.z, b.x, b.x);
            sC[t] = make_float4(b.y, b.y, b.z, b.z);
            sM[t] = make_float2(mq, mq);
        }
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
        if constexpr (ILP == 2) {
            if (!diag) {
                const float2 nxh = make_float2(-I.xh[0], -I.xh[1]), nyh = make_float2(-I.yh[0], -I.yh[1]);
                const float2 nzh = make_float2(-I.zh[0], -I.zh[1]), nxl = make_float2(-I.xl[0], -I.xl[1]);
                const float2 nyl = make_float2(-I.yl[0], -I.yl[1]), nzl = make_float2(-I.zl[0], -I.zl[1]);
                const float2 e2 = make_float2(eps2, eps2);
                float2 qm = make_float2(wres[0], wres[1]);
#pragma unroll 4
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 A = sA[jj], B = sB[jj], C = sC[jj];
                    const float2 M = sM[jj];
                    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), nxh), __fadd2_rn(make_float2(B.z, B.w), nxl));
                    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), nyh), __fadd2_rn(make_float2(C.x, C.y), nyl));
                    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), nzh), __fadd2_rn(make_float2(C.z, C.w), nzl));
                    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                    const float2 q = __fmul2_rn(r2, M);
                    qm.x = fminf(qm.x, q.x);
                    qm.y = fminf(qm.y, q.y);
                }
                wres[0] = qm.x;
                wres[1] = qm.y;
                continue;
            }
        }
        // scalar loop (the diagonal tiles, or ILP != 2), from the duplicated layout
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 A = sA[jj], B = sB[jj], C = sC[jj];
            const float4 J0 = make_float4(A.x, A.z, B.x, 0.f);
            const float4 J1 = make_float4(B.z, C.x, C.z, sM[jj].x);
            if (diag) wmax_mixed_j<ILP, true>(J0, J1, I, eps2, j0 + jj, ipos, wres);
            else wmax_mixed_j<ILP, false>(J0, J1, I, eps2, 0, ipos, wres);
        }
    }
    // max_j m_j / r^3 = q_min^(-3/2) (0 without sources, infinite for a coincident pair)
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float y = rsqrtf(wres[k]);
        wres[k] = y * y * y;
    }
}

// Gradient pass, mixed precision.  wmax: per active particle, max_j m_j / r^3 at the same
// positions (NULL: no deferred terms); up to GRAD_SLOTS terms heavier than SLOT_FRACTION x
// wmax are recorded during the loop and summed in double-float after it.
template <int BS, int ILP, int TJ, bool SMEM_SLOTS = false>
__device__ __forceinline__ void grad_mixed_body(const float4 *__restrict__ irec,
                                                const float4 *__restrict__ jrec, int n_a, int n_s,
                                                int ibase, int jb, int je, int self_pass, double eps2d,
                                                const float *__restrict__ wmax, double (&res)[ILP][3])
{
    // the grid kernels (two particles a thread, slot columns in shared memory) stage the
    // sources duplicated for the packed loop; the single-CTA solver as the four records
    constexpr bool X2 = (ILP == 2) && SMEM_SLOTS;
    __shared__ float4 s0[X2 ? 1 : TJ], s1[X2 ? 1 : TJ], s2[X2 ? 1 : TJ], s3[X2 ? 1 : TJ];
    __shared__ float4 sG[X2 ? 8 : 1][X2 ? TJ : 1];
    const int tid = threadIdx.x;
    const float eps2 = (float)eps2d;
    GradMixedI<ILP> I;
    int ipos[ILP];
    float thr[ILP];
    std::conditional_t<SMEM_SLOTS, SmemSlots<ILP, BS>, BigSlots<ILP>> big;
    if constexpr (SMEM_SLOTS) {
        __shared__ int s_slot[GRAD_SLOTS * ILP * BS];
        big.col = s_slot + tid;
#pragma unroll
        for (int k = 0; k < ILP; ++k) big.n[k] = 0;
    } else {
        init_big(big, 0);
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + tid;
        ipos[k] = i;
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0, q3 = q0;
        thr[k] = INFINITY;
        if (i < n_a) {
            q0 = irec[i];
            q1 = irec[n_a + i];
            q2 = irec[2 * n_a + i];
            q3 = irec[3 * n_a + i];
            if (wmax) thr[k] = SLOT_FRACTION * wmax[i];
        }
        I.xh[k] = q0.x; I.yh[k] = q0.y; I.zh[k] = q0.z;
        I.xm[k] = q1.x; I.ym[k] = q1.y; I.zm[k] = q1.z; I.ahx[k] = q1.w;
        I.xl[k] = q2.x; I.yl[k] = q2.y; I.zl[k] = q2.z; I.ahy[k] = q2.w;
        I.ahz[k] = q3.x; I.alx[k] = q3.y; I.aly[k] = q3.z; I.alz[k] = q3.w;
    }
    float hx[ILP], hy[ILP], hz[ILP], lx[ILP], ly[ILP], lz[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.f;

    if constexpr (X2) {
        GradX2I P;
        P.nxh = make_float2(-I.xh[0], -I.xh[1]);
        P.nyh = make_float2(-I.yh[0], -I.yh[1]);
        P.nzh = make_float2(-I.zh[0], -I.zh[1]);
        P.nxm = make_float2(-I.xm[0], -I.xm[1]);
        P.nym = make_float2(-I.ym[0], -I.ym[1]);
        P.nzm = make_float2(-I.zm[0], -I.zm[1]);
        P.nxl = make_float2(-I.xl[0], -I.xl[1]);
        P.nyl = make_float2(-I.yl[0], -I.yl[1]);
        P.nzl = make_float2(-I.zl[0], -I.zl[1]);
        P.nahx = make_float2(-I.ahx[0], -I.ahx[1]);
        P.nahy = make_float2(-I.ahy[0], -I.ahy[1]);
        P.nahz = make_float2(-I.ahz[0], -I.ahz[1]);
        P.nalx = make_float2(-I.alx[0], -I.alx[1]);
        P.naly = make_float2(-I.aly[0], -I.aly[1]);
        P.nalz = make_float2(-I.alz[0], -I.alz[1]);
        const float2 e2 = make_float2(eps2, eps2);
        const float (&thr2)[2] = *reinterpret_cast<const float(*)[2]>(thr);
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
                const float4 q0 = jrec[j0 + t], q1 = jrec[n_s + j0 + t];
                const float4 q2 = jrec[2 * n_s + j0 + t], q3 = jrec[3 * n_s + j0 + t];
                sG[0][t] = make_float4(q0.x, q0.x, q0.y, q0.y);
                sG[1][t] = make_float4(q0.z, q0.z, q1.x, q1.x);
                sG[2][t] = make_float4(q1.y, q1.y, q1.z, q1.z);
                sG[3][t] = make_float4(q2.x, q2.x, q2.y, q2.y);
                sG[4][t] = make_float4(q2.z, q2.z, q1.w, q1.w);
                sG[5][t] = make_float4(q2.w, q2.w, q3.x, q3.x);
                sG[6][t] = make_float4(q3.y, q3.y, q3.z, q3.z);
                sG[7][t] = make_float4(q3.w, q3.w, q0.w, q0.w);
            }
            __syncthreads();
            const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
            for (int c0 = 0; c0 < cnt; c0 += 64) {
                const int c1 = min(cnt, c0 + 64);
                float2 gx2 = make_float2(0.f, 0.f), gy2 = gx2, gz2 = gx2;
                if (!diag) {
                    int jj = c0;
                    for (; jj + 4 <= c1; jj += 4) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            grad_x2_j(sG[0][jj + u], sG[1][jj + u], sG[2][jj + u], sG[3][jj + u], sG[4][jj + u],
                                      sG[5][jj + u], sG[6][jj + u], sG[7][jj + u], P, e2, j0 + jj + u, thr2, big,
                                      gx2, gy2, gz2);
                    }
                    for (; jj < c1; ++jj)
                        grad_x2_j(sG[0][jj], sG[1][jj], sG[2][jj], sG[3][jj], sG[4][jj], sG[5][jj], sG[6][jj],
                                  sG[7][jj], P, e2, j0 + jj, thr2, big, gx2, gy2, gz2);
                } else {
                    // the i = j term masked by list position: the scalar body on the four records
                    float gx[ILP] = {0.f, 0.f}, gy[ILP] = {0.f, 0.f}, gz[ILP] = {0.f, 0.f};
                    for (int jj = c0; jj < c1; ++jj) {
                        const float4 G0 = sG[0][jj], G1 = sG[1][jj], G2 = sG[2][jj], G3 = sG[3][jj];
                        const float4 G4 = sG[4][jj], G5 = sG[5][jj], G6 = sG[6][jj], G7 = sG[7][jj];
                        const float4 J0 = make_float4(G0.x, G0.z, G1.x, G7.z);
                        const float4 J1 = make_float4(G1.z, G2.x, G2.z, G4.z);
                        const float4 J2 = make_float4(G3.x, G3.z, G4.x, G5.x);
                        const float4 J3 = make_float4(G5.z, G6.x, G6.z, G7.x);
                        grad_mixed_j<ILP, true>(J0, J1, J2, J3, I, eps2, j0 + jj, j0 + jj, ipos, thr, big, gx, gy,
                                                gz);
                    }
                    gx2 = make_float2(gx[0], gx[1]);
                    gy2 = make_float2(gy[0], gy[1]);
                    gz2 = make_float2(gz[0], gz[1]);
                }
                fold2(hx[0], lx[0], gx2.x);
                fold2(hy[0], ly[0], gy2.x);
                fold2(hz[0], lz[0], gz2.x);
                fold2(hx[1], lx[1], gx2.y);
                fold2(hy[1], ly[1], gy2.y);
                fold2(hz[1], lz[1], gz2.y);
            }
        }
    } else {
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            s0[t] = jrec[j0 + t];
            s1[t] = jrec[n_s + j0 + t];
            s2[t] = jrec[2 * n_s + j0 + t];
            s3[t] = jrec[3 * n_s + j0 + t];
        }
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
        for (int c0 = 0; c0 < cnt; c0 += 64) {
            const int c1 = min(cnt, c0 + 64);
            float gx[ILP], gy[ILP], gz[ILP];
#pragma unroll
            for (int k = 0; k < ILP; ++k) gx[k] = gy[k] = gz[k] = 0.f;
            int jj = c0;
            if (!diag) {
                for (; jj + 4 <= c1; jj += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        grad_mixed_j<ILP, false>(s0[jj + u], s1[jj + u], s2[jj + u], s3[jj + u], I, eps2,
                                                 j0 + jj + u, 0, ipos, thr, big, gx, gy, gz);
                }
                for (; jj < c1; ++jj)
                    grad_mixed_j<ILP, false>(s0[jj], s1[jj], s2[jj], s3[jj], I, eps2, j0 + jj, 0, ipos, thr,
                                             big, gx, gy, gz);
            } else {
                for (; jj < c1; ++jj)
                    grad_mixed_j<ILP, true>(s0[jj], s1[jj], s2[jj], s3[jj], I, eps2, j0 + jj, j0 + jj, ipos,
                                            thr, big, gx, gy, gz);
            }
#pragma unroll
            for (int k = 0; k < ILP; ++k) {
                fold2(hx[k], lx[k], gx[k]);
                fold2(hy[k], ly[k], gy[k]);
                fold2(hz[k], lz[k], gz[k]);
            }
        }
    }
    }
    // deferred double-float terms, records read back from global memory (L2)
    if constexpr (SMEM_SLOTS && BS == 32) {
        // the one-warp (small-tile) layout: shared by the lanes; the owner's records from irec
        double b[ILP][3];
#pragma unroll
        for (int k = 0; k < ILP; ++k) b[k][0] = b[k][1] = b[k][2] = 0.0;
        __shared__ D3 s_xbuf[BS];
        __syncwarp();
        warp_slot_terms<ILP>(big.n, s_xbuf, b, [&](int ol, int k, int s) -> D3 {
            const int j = big.col[(s * ILP + k) * BS + ol - tid];
            const int i = ibase + k * BS + ol;
            const float4 q0 = irec[i], q1 = irec[n_a + i], q2 = irec[2 * n_a + i], q3 = irec[3 * n_a + i];
            GradMixedI<1> O;
            O.xh[0] = q0.x; O.yh[0] = q0.y; O.zh[0] = q0.z;
            O.xm[0] = q1.x; O.ym[0] = q1.y; O.zm[0] = q1.z; O.ahx[0] = q1.w;
            O.xl[0] = q2.x; O.yl[0] = q2.y; O.zl[0] = q2.z; O.ahy[0] = q2.w;
            O.ahz[0] = q3.x; O.alx[0] = q3.y; O.aly[0] = q3.z; O.alz[0] = q3.w;
            D3 t = {0.0, 0.0, 0.0};
            grad_term_df<1>(jrec[j], jrec[n_s + j], jrec[2 * n_s + j], jrec[3 * n_s + j], O, 0, eps2d, t.x, t.y,
                            t.z);
            return t;
        });
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            res[k][0] = ((double)hx[k] + (double)lx[k]) + b[k][0];
            res[k][1] = ((double)hy[k] + (double)ly[k]) + b[k][1];
            res[k][2] = ((double)hz[k] + (double)lz[k]) + b[k][2];
        }
    } else {
        // per thread, summed in double-float
        const df::dfloat e2 = df::from_double(eps2d);
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            DF3 b = df3_zero();
            double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int s = 0; s < GRAD_SLOTS; ++s) {
                if (s < big.n[k]) {
                    const int j = big.get(s, k);
                    const float4 J0 = jrec[j], J1 = jrec[n_s + j], J2 = jrec[2 * n_s + j], J3 = jrec[3 * n_s + j];
                    DF3 t;
                    if (grad_term_df3<ILP>(J0, J1, J2, J3, I, k, e2, t)) df3_add(b, t);
                    else grad_term_fp64<ILP>(J0, J1, J2, J3, I, k, eps2d, f[0], f[1], f[2]);
                }
            }
            res[k][0] = ((double)hx[k] + (double)lx[k]) + (df::to_double(b.x) + f[0]);
            res[k][1] = ((double)hy[k] + (double)ly[k]) + (df::to_double(b.y) + f[1]);
            res[k][2] = ((double)hz[k] + (double)lz[k]) + (df::to_double(b.z) + f[2]);
        }
    }
}

// Time-step pass, mixed precision: best[k] = min_j min(t_ff s, t_fb s) (without eta),
// minr2[k] = min_j r^2 over the other particles
template <int BS, int ILP, int TJ, int SYM>
__device__ __forceinline__ void tstep_mixed_body(const float4 *__restrict__ irec,
                                                 const float4 *__restrict__ jrec, int n_a, int n_s,
                                                 int ibase, int jb, int je, int self_pass, float eta,
                                                 float (&best)[ILP], float (&minr2)[ILP])
{
    // two particles a thread: sources staged duplicated for the packed loop
    constexpr bool X2 = (ILP == 2);
    constexpr int TA = (SYM & 4) ? TJ : 1;
    __shared__ float4 s0[X2 ? 1 : TJ], s1[X2 ? 1 : TJ], sv[X2 ? 1 : TJ], sa[X2 ? 1 : TA];
    __shared__ float4 sA[X2 ? TJ : 1], sB[X2 ? TJ : 1], sC[X2 ? TJ : 1], sV0[X2 ? TJ : 1], sV1[X2 ? TJ : 1];
    __shared__ float4 sW0[X2 ? TA : 1], sW1[X2 ? TA : 1];
    const int tid = threadIdx.x;
    TstepMixedI<ILP> I;
    int ipos[ILP];
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const int i = ibase + k * BS + tid;
        ipos[k] = i;
        float4 a = make_float4(0.f, 0.f, 0.f, 1.f), b = make_float4(0.f, 0.f, 0.f, 0.f), c = a, d = b;
        if (i < n_a) {
            a = irec[i];
            b = irec[n_a + i];
            c = irec[2 * n_a + i];
            if (SYM & 4) d = irec[3 * n_a + i];
        }
        I.xh[k] = a.x; I.yh[k] = a.y; I.zh[k] = a.z;
        I.xl[k] = b.x; I.yl[k] = b.y; I.zl[k] = b.z;
        I.vx[k] = c.x; I.vy[k] = c.y; I.vz[k] = c.z; I.gm[k] = c.w;
        I.ax[k] = d.x; I.ay[k] = d.y; I.az[k] = d.z;
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) best[k] = minr2[k] = INFINITY;
    const float eta15 = 1.5f * eta;
    if constexpr (X2) {
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
        float (&best2)[2] = *reinterpret_cast<float(*)[2]>(best);
        float (&minr22)[2] = *reinterpret_cast<float(*)[2]>(minr2);
        float bnd[2] = {INFINITY, INFINITY}, ce[2] = {INFINITY, INFINITY};
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
                const float4 a = jrec[j0 + t], b = jrec[n_s + j0 + t], v = jrec[2 * n_s + j0 + t];
                sA[t] = make_float4(a.x, a.x, a.y, a.y);
                sB[t] = make_float4(a.z, a.z, b.x, b.x);
                sC[t] = make_float4(b.y, b.y, b.z, b.z);
                sV0[t] = make_float4(v.x, v.x, v.y, v.y);
                sV1[t] = make_float4(v.z, v.z, v.w, v.w);
                if (SYM & 4) {
                    const float4 w = jrec[3 * n_s + j0 + t];
                    sW0[t] = make_float4(w.x, w.x, w.y, w.y);
                    sW1[t] = make_float4(w.z, w.z, 0.f, 0.f);
                }
            }
            __syncthreads();
            const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
            if (!diag) {
                int jj = 0;
                for (; jj + 4 <= cnt; jj += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        tstep_x2_j<SYM>(sA[jj + u], sB[jj + u], sC[jj + u], sV0[jj + u], sV1[jj + u],
                                        (SYM & 4) ? sW0[jj + u] : zero4, (SYM & 4) ? sW1[jj + u] : zero4, P, eta,
                                        eta15, best2, minr22, bnd, ce);
                }
                for (; jj < cnt; ++jj)
                    tstep_x2_j<SYM>(sA[jj], sB[jj], sC[jj], sV0[jj], sV1[jj], (SYM & 4) ? sW0[jj] : zero4,
                                    (SYM & 4) ? sW1[jj] : zero4, P, eta, eta15, best2, minr22, bnd, ce);
            } else {
                // the i = j pair masked by list position: the scalar body on rebuilt records
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 a = sA[jj], b = sB[jj], c = sC[jj], v0 = sV0[jj], v1 = sV1[jj];
                    const float4 J0 = make_float4(a.x, a.z, b.x, 0.f);
                    const float4 J1 = make_float4(b.z, c.x, c.z, 0.f);
                    const float4 JV = make_float4(v0.x, v0.z, v1.x, v1.z);
                    float4 JA = zero4;
                    if (SYM & 4) JA = make_float4(sW0[jj].x, sW0[jj].z, sW1[jj].x, 0.f);
                    tstep_mixed_j<ILP, SYM, true>(J0, J1, JV, JA, I, eta, eta15, j0 + jj, ipos, best, minr2);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    bnd[k] = 1.001f * best[k];
                    ce[k] = bnd[k] * eta;
                }
            }
        }
    } else {
        for (int j0 = jb; j0 < je; j0 += TJ) {
            const int cnt = min(TJ, je - j0);
            __syncthreads();
            for (int t = tid; t < cnt; t += BS) {
                s0[t] = jrec[j0 + t];
                s1[t] = jrec[n_s + j0 + t];
                sv[t] = jrec[2 * n_s + j0 + t];
                if (SYM & 4) sa[t] = jrec[3 * n_s + j0 + t];
            }
            __syncthreads();
            const bool diag = self_pass && (j0 < ibase + BS * ILP) && (ibase < j0 + cnt);
            int jj = 0;
            if (!diag) {
                for (; jj + 4 <= cnt; jj += 4) {
    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        tstep_mixed_j<ILP, SYM, false>(s0[jj + u], s1[jj + u], sv[jj + u],
                                                       (SYM & 4) ? sa[jj + u] : zero4, I, eta, eta15, 0, ipos,
                                                       best, minr2);
                }
                for (; jj < cnt; ++jj)
                    tstep_mixed_j<ILP, SYM, false>(s0[jj], s1[jj], sv[jj], (SYM & 4) ? sa[jj] : zero4, I, eta, eta15,
                                                   0, ipos, best, minr2);
            } else {
                for (; jj < cnt; ++jj)
                    tstep_mixed_j<ILP, SYM, true>(s0[jj], s1[jj], sv[jj], (SYM & 4) ? sa[jj] : zero4, I, eta, eta15,
                                                  j0 + jj, ipos, best, minr2);
            }
        }
    }
}

// Newtonian pass, FP64 (one active particle per thread)
template <int BS, int TJ>
__device__ __forceinline__ void acc_fp64_body(const double4_32a *__restrict__ irec,
                                              const double4_32a *__restrict__ jrec, int n_a, int n_s,
                                              int ibase, int jb, int je, int self_pass, double eps2,
                                              double (&res)[3])
{
    __shared__ double4_32a s0[TJ];
    const int tid = threadIdx.x;
    const int i = ibase + tid;
    const double4_32a I = (i < n_a) ? irec[i] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) s0[t] = jrec[j0 + t];
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS) && (ibase < j0 + cnt);
        int jj = 0;
        if (!diag) {
            for (; jj + 4 <= cnt; jj += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc_fp64_j<false>(s0[jj + u], I, eps2, 0, i, ax, ay, az);
            }
            for (; jj < cnt; ++jj) acc_fp64_j<false>(s0[jj], I, eps2, 0, i, ax, ay, az);
        } else {
            for (; jj < cnt; ++jj) acc_fp64_j<true>(s0[jj], I, eps2, j0 + jj, i, ax, ay, az);
        }
    }
    res[0] = ax;
    res[1] = ay;
    res[2] = az;
}

// Gradient pass, FP64
template <int BS, int TJ>
__device__ __forceinline__ void grad_fp64_body(const double4_32a *__restrict__ irec,
                                               const double4_32a *__restrict__ jrec, int n_a, int n_s,
                                               int ibase, int jb, int je, int self_pass, double eps2,
                                               double (&res)[3])
{
    __shared__ double4_32a s0[TJ], s1[TJ];
    const int tid = threadIdx.x;
    const int i = ibase + tid;
    double4_32a I = make_double4_32a(0.0, 0.0, 0.0, 0.0), IA = I;
    if (i < n_a) {
        I = irec[i];
        IA = irec[n_a + i];
    }
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            s0[t] = jrec[j0 + t];
            s1[t] = jrec[n_s + j0 + t];
        }
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS) && (ibase < j0 + cnt);
        if (!diag) {
            for (int jj = 0; jj < cnt; ++jj) grad_fp64_j<false>(s0[jj], s1[jj], I, IA, eps2, 0, i, gx, gy, gz);
        } else {
            for (int jj = 0; jj < cnt; ++jj)
                grad_fp64_j<true>(s0[jj], s1[jj], I, IA, eps2, j0 + jj, i, gx, gy, gz);
        }
    }
    res[0] = gx;
    res[1] = gy;
    res[2] = gz;
}

// Time-step pass, FP64
template <int BS, int TJ, int SYM>
__device__ __forceinline__ void tstep_fp64_body(const double4_32a *__restrict__ irec,
                                                const double4_32a *__restrict__ jrec, int n_a, int n_s,
                                                int ibase, int jb, int je, int self_pass, double eta,
                                                double &best, double &minr2)
{
    __shared__ double4_32a s0[TJ], sv[TJ], sa[(SYM & 4) ? TJ : 1];
    const int tid = threadIdx.x;
    const int i = ibase + tid;
    const double4_32a zero4 = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    double4_32a I = make_double4_32a(0.0, 0.0, 0.0, 1.0), IV = make_double4_32a(0.0, 0.0, 0.0, 1.0), IA = zero4;
    if (i < n_a) {
        I = irec[i];
        IV = irec[n_a + i];
        if (SYM & 4) IA = irec[2 * n_a + i];
    }
    best = INFINITY;
    minr2 = INFINITY;
    for (int j0 = jb; j0 < je; j0 += TJ) {
        const int cnt = min(TJ, je - j0);
        __syncthreads();
        for (int t = tid; t < cnt; t += BS) {
            s0[t] = jrec[j0 + t];
            sv[t] = jrec[n_s + j0 + t];
            if (SYM & 4) sa[t] = jrec[2 * n_s + j0 + t];
        }
        __syncthreads();
        const bool diag = self_pass && (j0 < ibase + BS) && (ibase < j0 + cnt);
        if (!diag) {
            for (int jj = 0; jj < cnt; ++jj)
                tstep_fp64_j<SYM, false>(s0[jj], sv[jj], (SYM & 4) ? sa[jj] : zero4, I, IV, IA, eta, 0, i, best,
                                         minr2);
        } else {
            for (int jj = 0; jj < cnt; ++jj)
                tstep_fp64_j<SYM, true>(s0[jj], sv[jj], (SYM & 4) ? sa[jj] : zero4, I, IV, IA, eta, j0 + jj, i,
                                        best, minr2);
        }
    }
}

}  // namespace dev
}  // namespace frost
