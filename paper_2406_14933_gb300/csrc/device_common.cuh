// device_common.cuh -- device helpers shared by the step kernels: compensated
// accumulation, the per-edge terms of the scheme, boundary edges, the device-side
// time-step control (prepare / finish) and the end-of-step reduction.
//
// Scheme: Sec. 2.2, Eq. fvm_2D_eq_frac.07 in the fractional form of Appendix A.
#pragma once

#include <cfloat>
#include <cmath>

#include "asx_internal.cuh"

namespace asx {
namespace {

constexpr float kS32 = 0.866025403784438647f;     // sqrt(3) / 2

// ----------------------------------------------------------------- small helpers

// Error-free transformation a + b = s + e (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Adds x to the compensated pair (hi, lo) (lo collects the rounding errors).
__device__ __forceinline__ void acc_add(float &hi, float &lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// A compensated float32 pair used for per-thread ledger sums (boundary outflow, clamped
// water), so the per-cell path issues no float64 instruction; converted once per thread.
struct FF {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) { acc_add(hi, lo, x); }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Single-instruction approximations (PTX sqrt.approx / rcp.approx, relative error of a
// few ulp).  They only enter the friction solve and the wave speed, never the mass.
__device__ __forceinline__ float fast_sqrt(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// |(g1, g2)| without underflow of the squares for tiny momenta (rescaled when the sum of
// squares falls below the normal range).
__device__ __forceinline__ float norm2(float g1, float g2)
{
    const float q = __fmaf_rn(g1, g1, __fmul_rn(g2, g2));
    if (q >= 1.0e-36f) return fast_sqrt(q);
    const float s = fmaxf(fabsf(g1), fabsf(g2));
    if (s == 0.0f) return 0.0f;
    const float r = fast_rcp(s);
    const float a = g1 * r, b = g2 * r;
    return s * fast_sqrt(__fmaf_rn(a, a, b * b));
}

// Wave speed c = |v| + sqrt(g h) (Eq. fvm_2D_eq_frac.13) from the float32 state.
__device__ __forceinline__ float wave_speed(float v1, float v2, float h, float g)
{
    return __fadd_rn(fast_sqrt(__fmaf_rn(v1, v1, __fmul_rn(v2, v2))), fast_sqrt(__fmul_rn(g, h)));
}

// Bits of a wave speed for an unsigned max.  A wave speed is a sum of square roots, so
// it is +0, positive, +Inf or NaN; as unsigned integers these order like the floats, and
// a NaN of either sign sorts above +Inf, so a non-finite state reaches the step's c_max.
__device__ __forceinline__ unsigned speed_bits(float c)
{
    return __float_as_uint(c);
}

// Piecewise-linear rain rate r(t) [m/s], zero outside the table (Appendix C).
__device__ double rain_rate(const DevCtl *c, double t)
{
    const int n = c->n_rain;
    if (n <= 0) return 0.0;
    if (t < c->rain_t[0] || t > c->rain_t[n - 1]) return 0.0;
    if (n == 1) return c->rain_r[0];
    for (int k = 0; k + 1 < n; k++) {
        const double t0 = c->rain_t[k], t1 = c->rain_t[k + 1];
        if (t <= t1) {
            if (t1 == t0) return c->rain_r[k + 1];
            return c->rain_r[k] + (c->rain_r[k + 1] - c->rain_r[k]) * (t - t0) / (t1 - t0);
        }
    }
    return c->rain_r[n - 1];
}

// dt_n = min(dt_max, CFL phi / c_max^n), cut at t_end and the next sample time
// (Eqs. fvm_2D_eq_frac.12-13); fills the per-step scalars every CTA reads.
__device__ void prepare_step(DevCtl *c)
{
    c->active = 0;
    c->dt = 0.0;
    if (c->err) return;
    if (!(c->t < c->t_end) || c->step >= c->step_limit) return;
    double dt = c->dt_max;
    const double cmx = c->fp64 ? c->cmax64_cur : (double)c->cmax_cur;
    if (cmx > 0.0) {
        const double tau = c->cfl * c->phi / cmx;
        if (tau < dt) dt = tau;
    }
    double t_stop = c->t_end;
    if (c->sample_dt > 0.0) {
        const double ns = (double)(c->n_samples + 1) * c->sample_dt;
        if (ns < t_stop) t_stop = ns;
    }
    double tn;
    if (c->t + dt >= t_stop) {
        dt = t_stop - c->t;
        tn = t_stop;
    } else {
        tn = c->t + dt;
    }
    const double r = rain_rate(c, tn);
    c->dt = dt;
    c->t_next = tn;
    c->kappa = (float)(dt / c->sigma);
    c->qr = (float)(dt * r);
    c->qr64 = dt * r;
    c->dtf = (float)dt;
    c->active = 1;
}

// Adds a CTA's partial x to an order-independent sum: x = h 2^-30 + l 2^-70 (+ a rounding
// of at most 2^-71), h and l integers added with integer atomics, which commute exactly.
// |x| < 2^33 per partial; the fine part of one partial is below 2^40 units.
__device__ __forceinline__ void fx_add(unsigned long long *acc, double x)
{
    const double h = rint(x * 0x1p30);
    const double rem = fma(-h, 0x1p-30, x);          // exact: x - h 2^-30
    atomicAdd(&acc[0], (unsigned long long)(long long)h);
    atomicAdd(&acc[1], (unsigned long long)__double2ll_rn(rem * 0x1p70));
}

__device__ __forceinline__ double fx_value(const volatile unsigned long long *acc)
{
    return (double)(long long)acc[0] * 0x1p-30 + (double)(long long)acc[1] * 0x1p-70;
}

// Books the finished step (run by one thread after every CTA of the step is done).
__device__ void finish_step(DevCtl *c)
{
    volatile DevCtl *vc = c;
    const unsigned bits = vc->cmax_bits;
    const double outq = fx_value(vc->out_fx);
    const double clq = fx_value(vc->clamp_fx);
    const float cmax = __uint_as_float(bits);
    const double cmax64 = __longlong_as_double((long long)vc->cmax64_bits);
    c->rain_in += c->sigma * (double)c->ncells * (c->fp64 ? c->qr64 : (double)c->qr);
    c->outflow += c->sigma * outq;
    c->clamped += c->sigma * clq;
    c->t = c->t_next;
    c->step += 1;
    c->parity ^= 1;
    if (c->sample_dt > 0.0 && c->t == (double)(c->n_samples + 1) * c->sample_dt) {
        if (c->n_samples < c->max_samples) c->samples[c->n_samples] = c->outflow;
        c->n_samples += 1;
    }
    if (c->fp64) {
        if (!(cmax64 <= DBL_MAX)) c->err |= kErrNumeric;
        c->cmax64_cur = cmax64;
        c->cmax64_bits = 0ull;
    } else {
        if (!(cmax <= FLT_MAX)) c->err |= kErrNumeric;   // NaN or Inf somewhere
        c->cmax_cur = cmax;
    }
    c->cmax_bits = 0u;
    c->out_fx[0] = c->out_fx[1] = 0ull;
    c->clamp_fx[0] = c->clamp_fx[1] = 0ull;
    c->done_ctas = 0u;
    prepare_step(c);
}

// --------------------------------------------------------------- cell and edge terms

struct Cell {
    float m;    // theta*h (hi word)
    float v1, v2;
    float z;
    float h;    // m / theta
};

__device__ __forceinline__ float cell_theta(const StepArgs &a, size_t k)
{
    return a.cls ? a.cls_theta[a.cls[k]] : a.theta[k];
}

// 1 / theta of a cell: the class table's value, or one reciprocal instruction.  Every
// kernel forms the depth of a cell as h = (theta h) * (1 / theta) with this value, so a
// cell's depth is the same bits wherever it is evaluated.
__device__ __forceinline__ float cell_rtheta(const StepArgs &a, size_t k)
{
    return a.cls ? a.cls_rth[__ldg(a.cls + k)] : fast_rcp(__ldg(a.theta + k));
}

// Loads of the state planes in the per-cell code.  A step kernel that runs one step per
// launch reads state no other thread writes during the launch, so the read-only data
// path (ld.global.nc) is safe; a translation unit whose kernels run many steps in one
// launch (the ensemble) defines ASX_STATE_COHERENT_LOADS, and the loads are ordinary,
// ordered after the other CTAs' stores of the previous step by the barrier between steps.
#ifndef ASX_LD_STATE
#ifdef ASX_STATE_COHERENT_LOADS
#define ASX_LD_STATE(p) (*(p))
#else
#define ASX_LD_STATE(p) __ldg(p)
#endif
#endif

__device__ __forceinline__ Cell load_cell(const StepArgs &a, const float *mhi, const float *v1,
                                          const float *v2, size_t k)
{
    Cell q;
    q.m = ASX_LD_STATE(mhi + k);
    q.v1 = ASX_LD_STATE(v1 + k);
    q.v2 = ASX_LD_STATE(v2 + k);
    q.z = __ldg(a.z + k);
    q.h = __fmul_rn(q.m, cell_rtheta(a, k));
    return q;
}

// Terms of the edge between A (lower index) and B, B lying in owned direction D of A
// (0 = E, 1 = NE, 2 = NW), with kl2 = dt / sigma * l / 2 and l4 = l / 4:
//   mass increment   q  = dt / sigma * l (theta h)_(A,B) (v_n)_(A,B)   (Eqs. fvm_2D_eq.04, .06)
//   momentum flux    fa = l (theta h)_(A,B) (v_n)_(A,B) (v_a)_(A,B)
//   pressure term    p  = -1/2 l g (w_B - w_A) (theta h)^_(A,B) n_a     (Eq. fvm_2D_eq.05)
// (Eq. fvm_2D_eq_frac.01).  A receives -q, p - fa; B receives +q, p + fa.
// The terms of edge (A, B) that do not depend on the direction's normal components:
// q and fa as above and dh = (w_B - w_A)/g (theta h)^_(A,B), so that p = c dh with
// c = -1/2 l g n_a (c1, c2 per direction).
template <int D>
__device__ __forceinline__ void edge_core(const Cell &A, const Cell &B, float kl2, float l4, float &q, float &fa1,
                                          float &fa2, float &dh)
{
    const float s1 = __fadd_rn(A.v1, B.v1);          // 2 (v_1)_(A,B)
    const float s2 = __fadd_rn(A.v2, B.v2);
    float vn2;                                       // 2 (v_n)_(A,B)
    if (D == 0) vn2 = s1;
    else if (D == 1) vn2 = __fmaf_rn(kS32, s2, __fmul_rn(0.5f, s1));
    else vn2 = __fmaf_rn(kS32, s2, __fmul_rn(-0.5f, s1));
    // the upwind theta h depends on v_n alone (any side if v_n = 0), so the mass
    // increment does not wait for the surface difference
    const float mu = vn2 > 0.0f ? A.m : B.m;
    const float G = __fmul_rn(mu, vn2);
    q = __fmul_rn(kl2, G);
    const float gl = __fmul_rn(l4, G);
    fa1 = __fmul_rn(gl, s1);
    fa2 = __fmul_rn(gl, s2);
    const float dw = __fadd_rn(__fsub_rn(B.z, A.z), __fsub_rn(B.h, A.h));   // (w_B - w_A) / g
    const float hat = vn2 != 0.0f ? mu : (dw < 0.0f ? A.m : B.m);           // tie: higher surface
    dh = __fmul_rn(dw, hat);
}

template <int D>
__device__ __forceinline__ void edge_terms(const Cell &A, const Cell &B, float kl2, float l4,
                                           float c1, float c2, float &q, float &fa1, float &fa2,
                                           float &p1, float &p2)
{
    float dh;
    edge_core<D>(A, B, kl2, l4, q, fa1, fa2, dh);
    p1 = __fmul_rn(c1, dh);
    p2 = __fmul_rn(c2, dh);
}

// Artificial-viscosity coefficient of edge (A, B) (Appendix A, Eqs. eq_artif_visc,
// eq_visc1): t = l c_(A,B) mu_(A,B), c_(A,B) = max(c_A, c_B) with c = |v| + sqrt(g h),
// mu_(A,B) = 2 m_A m_B / (m_A + m_B) (0 when both are dry).  Symmetric in A and B bit
// for bit; cell A's momentum sum gains t (v_B - v_A), cell B's t (v_A - v_B).
__device__ __forceinline__ float visc_coef(const Cell &A, const Cell &B, float l, float g)
{
    const float c = fmaxf(wave_speed(A.v1, A.v2, A.h, g), wave_speed(B.v1, B.v2, B.h, g));
    const float den = __fadd_rn(A.m, B.m);
    const float mu = den > 1.0e-30f ? __fmul_rn(__fmul_rn(2.0f, __fmul_rn(A.m, B.m)), fast_rcp(den)) : 0.0f;
    return __fmul_rn(__fmul_rn(l, c), mu);
}

// Update of one cell once all its edge terms are in (Appendix A): rain at t^{n+1},
// clamp of a negative mass, theta h v^* = theta h^n v^n + dt / sigma (J + S), and the
// closed-form implicit friction v^{n+1} = 2 gamma / (alpha + sqrt(alpha^2 + 4 beta |gamma|))
// with alpha = theta h^{n+1}, beta = dt K(h^{n+1}, theta) (Eq. miu-formula).  Returns the
// new state, the bits of the new wave speed, and adds clamped mass to clq.  EXT: the
// optional linear resistance (dtau = dt tau) and dry threshold are compiled in; without
// them (callers that never set them) the code is the plain update.
struct CellNew {
    float hi, lo, v1, v2;
    unsigned cbits;
};

template <bool EXT = true>
__device__ __forceinline__ CellNew cell_update(float shi, float slo, float M1, float M2, float m_old,
                                               float v1_old, float v2_old, float rth, float ka, float kb,
                                               float kappa, float qr, float dtf, float g, float dtau,
                                               float h_dry, FF &clq)
{
    CellNew o;
    acc_add(shi, slo, qr);
    float hi, lo;
    two_sum(shi, slo, hi, lo);
    if (hi < 0.0f || (hi == 0.0f && lo < 0.0f)) {
        clq.add(-hi);
        clq.add(-lo);
        hi = 0.0f;
        lo = 0.0f;
    }
    const float g1 = __fmaf_rn(kappa, M1, __fmul_rn(m_old, v1_old));
    const float g2 = __fmaf_rn(kappa, M2, __fmul_rn(m_old, v2_old));
    const float h = __fmul_rn(hi, rth);
    const float beta = __fmul_rn(dtf, __fmaf_rn(ka, h, kb));
    const float ng = norm2(g1, g2);
    // a linear resistance -tau h v (Thacker's problem), implicit like the rest, adds
    // dt tau h^{n+1} to alpha (dtau = dt tau; 0 leaves alpha = theta h bit for bit)
    float ap = hi;
    if constexpr (EXT) ap = __fmaf_rn(dtau, h, hi);
    const float den = __fadd_rn(ap, fast_sqrt(__fmaf_rn(ap, ap, __fmul_rn(4.0f * beta, ng))));
    float w1 = 0.0f, w2 = 0.0f;
    if (den > 1.0e-30f) {
        const float inv2 = __fmul_rn(2.0f, fast_rcp(den));
        w1 = __fmul_rn(g1, inv2);
        w2 = __fmul_rn(g2, inv2);
    } else if (den > 0.0f) {
        // tiny or subnormal denominator: scale it (and the numerators) by 2^64 first
        const float inv2 = __fmul_rn(2.0f, fast_rcp(__fmul_rn(den, 0x1p64f)));
        w1 = __fmul_rn(__fmul_rn(g1, 0x1p64f), inv2);
        w2 = __fmul_rn(__fmul_rn(g2, 0x1p64f), inv2);
    }
    if constexpr (EXT) {
        if (h < h_dry) {         // optional dry threshold (0: none)
            w1 = 0.0f;
            w2 = 0.0f;
        }
    }
    o.hi = hi;
    o.lo = lo;
    o.v1 = w1;
    o.v2 = w2;
    o.cbits = speed_bits(wave_speed(w1, w2, h, g));
    return o;
}

// Boundary type at position pos along `side`: the side's type inside its interval
// [fb, fe) (all of it when fb == fe), a wall outside.
__device__ __forceinline__ int side_type(const StepArgs &a, int side, int pos)
{
    if (a.fb[side] == a.fe[side]) return a.bc[side];
    return (pos >= a.fb[side] && pos < a.fe[side]) ? a.bc[side] : ASX_BC_WALL;
}

// Neighbour of (r, c) in direction d (0 E, 1 NE, 2 NW, 3 W, 4 SW, 5 SE); odd rows are
// shifted east.  Returns false and the boundary side if it lies outside the raster.
__device__ __forceinline__ bool neighbour(int rows, int cols, int r, int c, int d, int &rr, int &cc,
                                          int &side)
{
    const int odd = r & 1;
    rr = r;
    cc = c;
    switch (d) {
    case 0: cc = c + 1; break;
    case 1: rr = r + 1; cc = c + odd; break;
    case 2: rr = r + 1; cc = c - 1 + odd; break;
    case 3: cc = c - 1; break;
    case 4: rr = r - 1; cc = c - 1 + odd; break;
    default: rr = r - 1; cc = c + odd; break;
    }
    if (rr < 0) { side = ASX_SIDE_S; return false; }
    if (rr >= rows) { side = ASX_SIDE_N; return false; }
    if (cc < 0) { side = ASX_SIDE_W; return false; }
    if (cc >= cols) { side = ASX_SIDE_E; return false; }
    return true;
}

__constant__ float kN1[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
__constant__ float kN2[6] = {0.0f, kS32, kS32, 0.0f, -kS32, -kS32};

// Free-discharge edge of cell X in direction d: a ghost copy of X, outflow only, so
// F = l (theta h)_X max(v_X . n, 0), momentum flux F v_X, no pressure term.  The
// increment is booked in outd exactly as applied.
__device__ __forceinline__ void free_edge(const Cell &X, int d, float kl2, float l2, float &shi,
                                          float &slo, float &M1, float &M2, FF &outd)
{
    const float vn2 = 2.0f * __fmaf_rn(X.v1, kN1[d], __fmul_rn(X.v2, kN2[d]));
    if (vn2 > 0.0f) {
        const float G = __fmul_rn(X.m, vn2);
        const float q = __fmul_rn(kl2, G);
        const float F = __fmul_rn(l2, G);
        acc_add(shi, slo, -q);
        M1 -= F * X.v1;
        M2 -= F * X.v2;
        outd.add(q);
    }
}

// Scalars of the pending step, read once per CTA.
struct StepScalars {
    int par;
    float kappa, qr, dtf, kl2, l4, l2;
};

__device__ __forceinline__ StepScalars step_scalars(const StepArgs &a)
{
    const DevCtl *ctl = a.ctl;
    StepScalars s;
    s.par = ctl->parity;
    s.kappa = ctl->kappa;
    s.qr = ctl->qr;
    s.dtf = ctl->dtf;
    s.kl2 = s.kappa * (0.5f * a.l);
    s.l4 = 0.25f * a.l;
    s.l2 = 0.5f * a.l;
    return s;
}

// Given-mass-flux edge of cell X in direction d on `side` (Sec. 3): the edge admits
// l q (n_side . n_d) per unit time, entering along the inward side normal with speed
// q / max(h, h_c), h_c = (q^2/g)^(1/3) the critical depth; no pressure term (the ghost's
// surface is the cell's).  The depth increment kappa l q (n_side . n_d) is booked in outd
// as negative outflow, exactly as applied.
__device__ __forceinline__ void flux_edge(const StepArgs &a, const Cell &X, int d, int side, float kappa,
                                          float &shi, float &slo, float &M1, float &M2, FF &outd)
{
    const float q = a.bq[side];
    if (!(q > 0.0f)) return;
    const float ns1 = side == ASX_SIDE_W ? -1.0f : side == ASX_SIDE_E ? 1.0f : 0.0f;
    const float ns2 = side == ASX_SIDE_S ? -1.0f : side == ASX_SIDE_N ? 1.0f : 0.0f;
    const float fin = __fmul_rn(__fmul_rn(a.l, q), __fmaf_rn(ns1, kN1[d], __fmul_rn(ns2, kN2[d])));
    const float qd = __fmul_rn(kappa, fin);
    const float mom = __fmul_rn(fin, __fdiv_rn(q, fmaxf(X.h, a.bhc[side])));
    acc_add(shi, slo, qd);
    M1 -= __fmul_rn(mom, ns1);
    M2 -= __fmul_rn(mom, ns2);
    outd.add(-qd);
}

// Dirichlet edge of cell X (stored at index k) in direction d on `side` (Sec. 4, Eq.
// numerics-bc): a ghost cell on X's bed and porosity with depth h_b and velocity
// -u_b n_side, through the interior edge function in its canonical orientation; the
// mass through the edge is booked in outd (outflow positive).
__device__ __forceinline__ void dirichlet_edge(const StepArgs &a, const StepScalars &s, const Cell &X, size_t k,
                                               int d, int side, float &shi, float &slo, float &M1, float &M2,
                                               FF &outd)
{
    const float ns1 = side == ASX_SIDE_W ? -1.0f : side == ASX_SIDE_E ? 1.0f : 0.0f;
    const float ns2 = side == ASX_SIDE_S ? -1.0f : side == ASX_SIDE_N ? 1.0f : 0.0f;
    Cell G;
    G.h = a.bh[side];
    G.m = __fmul_rn(cell_theta(a, k), G.h);
    G.v1 = __fmul_rn(-a.bu[side], ns1);
    G.v2 = __fmul_rn(-a.bu[side], ns2);
    G.z = X.z;
    float q, f1, f2, p1, p2;
    switch (d) {
    case 0: edge_terms<0>(X, G, s.kl2, s.l4, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
    case 1: edge_terms<1>(X, G, s.kl2, s.l4, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
    case 2: edge_terms<2>(X, G, s.kl2, s.l4, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
    case 3: edge_terms<0>(G, X, s.kl2, s.l4, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
    case 4: edge_terms<1>(G, X, s.kl2, s.l4, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
    default: edge_terms<2>(G, X, s.kl2, s.l4, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
    }
    if (d < 3) {                  // X is the lower cell: it loses q
        acc_add(shi, slo, -q);
        M1 += p1 - f1;
        M2 += p2 - f2;
        outd.add(q);
    } else {
        acc_add(shi, slo, q);
        M1 += p1 + f1;
        M2 += p2 + f2;
        outd.add(-q);
    }
}

// The whole step for one cell (r, c), gathering its six neighbours from global memory:
// each edge is evaluated in its canonical orientation (the lower cell first), so a
// shared edge gives both cells the same mass increment wherever it is evaluated.
// EXT: the optional terms (artificial viscosity, linear resistance, dry threshold) are
// compiled in; the ensemble, whose scenarios never set them, leaves them out.  BND: the
// inflow sides (given mass flux, Dirichlet) are compiled in.
template <bool EXT = true, bool BND = true>
__device__ __forceinline__ void gather_cell(const StepArgs &a, const StepScalars &s, int r, int c,
                                            unsigned &cb, FF &outd, FF &clq)
{
    const float *mhi = a.mhi[s.par], *mlo = a.mlo[s.par], *v1 = a.v1[s.par], *v2 = a.v2[s.par];
    const size_t k = (size_t)r * a.pitch + c;
    const Cell I = load_cell(a, mhi, v1, v2, k);
    float shi = I.m, slo = ASX_LD_STATE(mlo + k);
    float M1 = 0.0f, M2 = 0.0f;      // J_a + S_a
#pragma unroll
    for (int d = 0; d < 6; d++) {
        int rr, cc, side;
        if (neighbour(a.rows, a.cols, r, c, d, rr, cc, side)) {
            const Cell J = load_cell(a, mhi, v1, v2, (size_t)rr * a.pitch + cc);
            float q, f1, f2, p1, p2;
            switch (d) {
            case 0: edge_terms<0>(I, J, s.kl2, s.l4, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
            case 1: edge_terms<1>(I, J, s.kl2, s.l4, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
            case 2: edge_terms<2>(I, J, s.kl2, s.l4, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
            case 3: edge_terms<0>(J, I, s.kl2, s.l4, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
            case 4: edge_terms<1>(J, I, s.kl2, s.l4, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
            default: edge_terms<2>(J, I, s.kl2, s.l4, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
            }
            if (d < 3) {              // I is the lower cell: it loses q
                acc_add(shi, slo, -q);
                M1 += p1 - f1;
                M2 += p2 - f2;
            } else {
                acc_add(shi, slo, q);
                M1 += p1 + f1;
                M2 += p2 + f2;
            }
            if (EXT && a.visc) {
                const float t = visc_coef(I, J, a.l, a.g);
                M1 += __fmul_rn(t, __fsub_rn(J.v1, I.v1));
                M2 += __fmul_rn(t, __fsub_rn(J.v2, I.v2));
            }
        } else {
            const int pos = (side == ASX_SIDE_S || side == ASX_SIDE_N) ? c : r;
            const int bt = side_type(a, side, pos);
            if (bt == ASX_BC_FREE) free_edge(I, d, s.kl2, s.l2, shi, slo, M1, M2, outd);
            else if (BND && bt == ASX_BC_FLUX) flux_edge(a, I, d, side, s.kappa, shi, slo, M1, M2, outd);
            else if (BND && bt == ASX_BC_DIRICHLET) dirichlet_edge(a, s, I, k, d, side, shi, slo, M1, M2, outd);
            // wall: mirror ghost, the edge carries nothing
        }
    }
    float th, ka, kb, rth;
    if (a.cls) {
        const int cl = a.cls[k];
        th = a.cls_theta[cl];
        rth = a.cls_rth[cl];
        ka = a.cls_a[cl];
        kb = a.cls_b[cl];
    } else {
        th = a.theta[k];
        rth = fast_rcp(th);
        ka = a.alpha_p * (1.0f - th);
        kb = th * a.alpha_s;
    }
    const CellNew o = cell_update<EXT>(shi, slo, M1, M2, I.m, I.v1, I.v2, rth, ka, kb, s.kappa, s.qr, s.dtf,
                                  a.g, __fmul_rn(s.dtf, a.tau), a.h_dry, clq);
    const int np = s.par ^ 1;
    a.mhi[np][k] = o.hi;
    a.mlo[np][k] = o.lo;
    a.v1[np][k] = o.v1;
    a.v2[np][k] = o.v2;
    cb = max(cb, o.cbits);
}

// Block reduction of (max c, sum outflow, sum clamp) and the last-CTA step finish.
template <int NT>
__device__ __forceinline__ void reduce_and_finish(const StepArgs &a, unsigned cbits, double outq,
                                                  double clq)
{
    __shared__ unsigned s_max[NT / 32];
    __shared__ double s_out[NT / 32], s_cl[NT / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    unsigned bits = __reduce_max_sync(0xffffffffu, cbits);
    if (__any_sync(0xffffffffu, outq != 0.0 || clq != 0.0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            outq += __shfl_down_sync(0xffffffffu, outq, o);
            clq += __shfl_down_sync(0xffffffffu, clq, o);
        }
    }
    if (lane == 0) {
        s_max[wid] = bits;
        s_out[wid] = outq;
        s_cl[wid] = clq;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned mb = 0u;
        double so = 0.0, sc = 0.0;
        for (int w = 0; w < NT / 32; w++) {
            mb = max(mb, s_max[w]);
            so += s_out[w];
            sc += s_cl[w];
        }
        DevCtl *ctl = a.ctl;
        atomicMax(&ctl->cmax_bits, mb);
        if (so != 0.0) fx_add(ctl->out_fx, so);
        if (sc != 0.0) fx_add(ctl->clamp_fx, sc);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->done_ctas, 1u);
        s_last = (prev == (unsigned)a.nblocks - 1u);
        if (s_last) {
            __threadfence();
            finish_step(ctl);
        }
    }
}

}  // namespace

}  // namespace asx
