// strip_tile.cuh -- the strip tile worker of the main step kernel and of the strip
// ensemble kernel: one warp marches down a 128-column tile fed by TMA, four cells per
// lane, two at a time in the packed float32 pairs of sm_100+, plus the frame cells' gather
// loop.  Included by step_strip.cu and ensemble.cu; every definition has internal linkage.
//
// Same arithmetic as the gather kernel (Sec. 2.2, Eq. fvm_2D_eq_frac.07 in the form of
// Appendix A), organised for GB300:
//   * a tile worker is one warp and owns kSW = 128 columns x H rows (in the step kernel
//     the worker is a one-warp CTA, in the strip ensemble kernel a warp of a larger
//     CTA, with its own ring and mbarriers); lane L owns the cells at
//     columns c0 + 2L + e (left half of the tile) and c0 + 64 + 2L + e (right half),
//     e = 0, 1.  The two cells with the same e lie 64 columns apart in the same row and
//     see the same stencil: they form a float2 pair that the edge and cell code process
//     together with the f32x2 instructions (add / sub / mul / fma .rn.f32x2: one issue
//     slot for two float32 operations, each component rounded as the scalar operation);
//   * rows r0-1 .. r0+H of every field (one halo row above and below, halo columns left
//     and right) stream into a shared-memory ring of 2-row chunks through TMA tensor
//     loads (cp.async.bulk.tensor.2d) that complete on mbarriers; lane 0 refills a chunk
//     once every row of it is finished;
//   * the warp walks the tile row by row; the edges between row r and r+1 and the east
//     edges of row r are evaluated by the lane that owns their lower cell; a lane also
//     evaluates the one horizontal and one diagonal edge it shares with each neighbouring
//     lane (the same canonical edge, so the same bits), which replaces every exchange of
//     edge terms; every lane reads the cells beside its own (in its own row and the
//     next, including the halo columns at the tile ends) from the ring: the same values,
//     hence the same bits, as the neighbouring lane's own cells;
//   * contributions to row r+1 stay in registers until that row is finished; no block
//     barrier is needed;
//   * tiles are laid out so that each tile with its halo lies inside the raster, which
//     leaves no boundary edge in the tile code; the remaining cells along the raster
//     sides (the frame) are processed in the same launch by frame CTAs that gather each
//     cell's six neighbours (the same per-cell code as the gather kernel).
// Both cells of an edge accumulate the mass increment of the same canonical edge
// function, bit for bit the increment the scalar code of the frame computes, so opposite
// increments are identical and the water budget closes to float64 rounding.  The edge
// code works with the normal component scaled by +-2 (exact) and keeps the momentum sums
// in units of l/8, which saves a multiply and two constants per diagonal edge.  The cell
// update of a row runs without branches (cell_update_fast) for both pairs, so the code
// generator can interleave their long dependency chains; a clamp, a vanishing momentum or
// friction denominator, or a NaN sends the pair through the full update with its
// branches, which gives the same bits in every other case.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "device_common.cuh"

namespace asx {

namespace {

#ifndef ASX_STRIP_NC
#define ASX_STRIP_NC 2
#endif
#ifndef ASX_STRIP_MINB
#define ASX_STRIP_MINB 16
#endif
constexpr int kSW = kStripW;           // tile width in cells
constexpr int kRB = kStripChunkRows;   // rows per ring chunk (= TMA box height)
constexpr int kNC = ASX_STRIP_NC;      // chunks in the ring
constexpr int kBXF = kSW + 8;          // float box width (from column c0 - 4)
constexpr int kBXC = kSW + 16;         // uint8 box width (from column c0 - 4)
constexpr int kXO = 4;                 // ring x index of column c0 (float fields)
constexpr int kXOC = 4;                // ring x index of column c0 (class field)
// TMA tiled loads must start on a 16-byte boundary: every tile column c0 is 4 mod 128,
// so float boxes start at c0 - 4 (a multiple of 128 elements), the low-mass box at c0
// (16 bytes past a multiple of 512), and the uint8 class box at c0 - 4 (a multiple of
// 128 bytes).
static_assert(kXOC == kXO && (kBXC % 16) == 0 && ((kBXF * 4) % 16) == 0, "TMA box alignment");

constexpr int kFBoxBytes = (kRB * kBXF * 4 + 127) / 128 * 128;
struct __align__(128) FBox { float v[kRB][kBXF]; float pad[(kFBoxBytes - kRB * kBXF * 4) / 4]; };
struct __align__(128) LBox { float v[kRB][kSW]; };
struct __align__(128) CBox { uint8_t v[kRB][kBXC]; };
static_assert(sizeof(FBox) == kFBoxBytes && kFBoxBytes > kRB * kBXF * 4, "box padding");

// One ring chunk: kRB rows of every field; the porosity slot holds theta (float) or, in
// land-cover-class mode, the uint8 class ids.
template <bool CLS>
struct __align__(128) Chunk {
    FBox mhi, v1, v2, z;
    typename std::conditional<CLS, CBox, FBox>::type th;
    LBox mlo;
};

template <bool CLS>
struct StripSmem {
    Chunk<CLS> ring[kNC];
    unsigned long long bar[kNC];
};

// ----------------------------------------------------------------- bounds checks
//
// The bounds-checked debug build (-DASX_BOUNDS_CHECK, `build.build_checked`) tests every
// shared-memory ring index and global store of the tile code: an index outside its buffer
// sets kErrBounds in the step's error word (reported as ASX_EBOUNDS) and the access is
// skipped or redirected to element 0.  The ordinary build compiles no check.
#ifdef ASX_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(const StepArgs &a, long long i, long long n)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&a.ctl->err, kErrBounds);
    return false;
}
#define ASX_RING(a, i, n) (in_bounds((a), (i), (n)) ? (i) : 0)
#define ASX_STORE_OK(a, i, n) in_bounds((a), (i), (n))
#else
#define ASX_RING(a, i, n) (i)
#define ASX_STORE_OK(a, i, n) true
#endif

// ----------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Returns an mbarrier with no pending arrivals or copies to the uninitialised state, so
// that its word can be initialised again (a warp that runs several tiles with one ring).
__device__ __forceinline__ void mbar_inval(unsigned long long *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Makes a tensor map that the host wrote to global memory visible to the tensor-copy
// proxy of the calling thread (maps passed as kernel parameters need no fence).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase: each try_wait suspends the warp until the phase
// completes or a short hardware-defined interval passes; gives up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// ----------------------------------------------------------------- packed pairs

// The packed operations are written as PTX with an explicit rounding mode: like the
// scalar __fadd_rn / __fmul_rn, they are then never contracted into a fused multiply-add,
// which the error-free two-sums below depend on.
__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// two_sum on both components
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// (hi, lo) += x on both components, as acc_add
__device__ __forceinline__ void acc_add2(float2 &hi, float2 &lo, float2 x)
{
    float2 s, e;
    two_sum2(hi, x, s, e);
    hi = s;
    lo = add2(lo, e);
}

// (hi, lo) += -x with the bits of acc_add(hi, lo, -x): there b - bb = -x - bb rounds
// to -(x + bb)
__device__ __forceinline__ void acc_sub2(float2 &hi, float2 &lo, float2 x)
{
    const float2 s = sub2(hi, x);
    const float2 bb = sub2(s, hi);
    const float2 e = sub2(sub2(hi, sub2(s, bb)), add2(x, bb));
    hi = s;
    lo = add2(lo, e);
}

__device__ __forceinline__ float &comp(float2 &v, int s) { return s ? v.y : v.x; }
__device__ __forceinline__ float comp(const float2 &v, int s) { return s ? v.y : v.x; }

struct PCell {
    float2 m, v1, v2, z, h;
};

struct PAcc {
    float2 hi, lo, m1, m2;
};

__device__ __forceinline__ Cell half_cell(const PCell &P, int s)
{
    return Cell{comp(P.m, s), comp(P.v1, s), comp(P.v2, s), comp(P.z, s), comp(P.h, s)};
}

// Edge (X lower, Y upper) in direction D for both halves of the pairs, the terms of
// edge_core component by component; adds them to ax if ux and to ay if uy (a side not
// used belongs to another lane or is not updated by this tile).
//
// Scaled form.  u = 2 v_n for E and NE, u = -2 v_n for NW, where v_n is edge_core's
// normal component (itself twice the interface velocity's): scaling by a power of two is
// exact, so G = mu u is exactly +-2 edge_core's G and q = (kl2 / 2) G is exactly +-q of
// edge_core, the same bits in every normal-range case (a normal component or flux below
// 2^-126 may differ in its last subnormal bit, a mass of order 1e-45 of the cell's).  A
// NW edge's negative q enters the sums with the opposite operation (acc_add2(x) has the
// bits of acc_sub2(-x)).  The momentum sums are kept in units of l/8, so the flux terms
// are G s without a factor and the pressure coefficients are a.cpm = -4 g n; the cell
// update multiplies them by dt/sigma * l/8.  With EXT and a.visc the artificial viscosity
// adds t (v_Y - v_X) to X and t (v_X - v_Y) to Y, t scaled by vs = 8/l.
template <int D, bool EXT>
__device__ __forceinline__ void edge(const StepArgs &a, const PCell &X, const PCell &Y, float2 kh, float vs,
                                      PAcc &ax, bool ux, PAcc &ay, bool uy)
{
    constexpr float kSgn = D == 2 ? -1.0f : 1.0f;
    const float2 s1 = add2(X.v1, Y.v1), s2 = add2(X.v2, Y.v2);
    float2 u;
    if (D == 0) u = add2(s1, s1);
    else u = fma2(dup2(kSgn * 2.0f * kS32), s2, s1);
    const float2 dw = add2(sub2(Y.z, X.z), sub2(Y.h, X.h));
    // the upwind side is the sign of v_n, or at v_n = 0 that of -dw
    float2 mu;
    if (D != 2) {
        const float kx = u.x != 0.0f ? u.x : -dw.x, ky = u.y != 0.0f ? u.y : -dw.y;
        mu.x = kx > 0.0f ? X.m.x : Y.m.x;
        mu.y = ky > 0.0f ? X.m.y : Y.m.y;
    } else {
        const float kx = u.x != 0.0f ? u.x : dw.x, ky = u.y != 0.0f ? u.y : dw.y;
        mu.x = kx < 0.0f ? X.m.x : Y.m.x;
        mu.y = ky < 0.0f ? X.m.y : Y.m.y;
    }
    const float2 G = mul2(mu, u);
    // q = kh G as fma(kh, G, +0): the same bits as the product (but for the sign of a
    // zero, which moves no mass), and an instruction the code generator cannot fuse into
    // the two-sums that consume q, as it was seen to do with a plain packed multiply
    const float2 q = fma2(kh, G, dup2(0.0f));
    const float2 f1 = mul2(G, s1), f2 = mul2(G, s2);
    const float2 dh = mul2(dw, mu);
    // an E edge's normal has no second component: its pressure term leaves m2 as it is
    const float2 c1 = dup2(a.cpm[D][0]), c2 = dup2(a.cpm[D][1]);
    if (ux) {
        if (D != 2) {
            acc_sub2(ax.hi, ax.lo, q);
            ax.m1 = sub2(fma2(c1, dh, ax.m1), f1);
            ax.m2 = sub2(D == 0 ? ax.m2 : fma2(c2, dh, ax.m2), f2);
        } else {
            acc_add2(ax.hi, ax.lo, q);
            ax.m1 = add2(fma2(c1, dh, ax.m1), f1);
            ax.m2 = add2(fma2(c2, dh, ax.m2), f2);
        }
    }
    if (uy) {
        if (D != 2) {
            acc_add2(ay.hi, ay.lo, q);
            ay.m1 = add2(fma2(c1, dh, ay.m1), f1);
            ay.m2 = add2(D == 0 ? ay.m2 : fma2(c2, dh, ay.m2), f2);
        } else {
            acc_sub2(ay.hi, ay.lo, q);
            ay.m1 = sub2(fma2(c1, dh, ay.m1), f1);
            ay.m2 = sub2(fma2(c2, dh, ay.m2), f2);
        }
    }
    if (EXT && a.visc) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const Cell Xs = half_cell(X, s), Ys = half_cell(Y, s);
            const float t = __fmul_rn(visc_coef(Xs, Ys, a.l, a.g), vs);
            const float d1 = __fsub_rn(Ys.v1, Xs.v1), d2 = __fsub_rn(Ys.v2, Xs.v2);
            if (ux) {
                comp(ax.m1, s) = __fmaf_rn(t, d1, comp(ax.m1, s));
                comp(ax.m2, s) = __fmaf_rn(t, d2, comp(ax.m2, s));
            }
            if (uy) {
                comp(ay.m1, s) = __fmaf_rn(-t, d1, comp(ay.m1, s));
                comp(ay.m2, s) = __fmaf_rn(-t, d2, comp(ay.m2, s));
            }
        }
    }
}

// cell_update for both halves of a pair, component by component the same operations
// (the rare branches, a clamp or a tiny denominator, taken per component).
struct CellNew2 {
    float2 hi, lo, v1, v2;
    unsigned cb0, cb1;
};

__device__ __forceinline__ void tiny_den(float den, float g1, float g2, float &w1, float &w2)
{
    if (den > 0.0f) {
        // tiny or subnormal denominator: scale it (and the numerators) by 2^64 first
        const float inv2 = __fmul_rn(2.0f, fast_rcp(__fmul_rn(den, 0x1p64f)));
        w1 = __fmul_rn(__fmul_rn(g1, 0x1p64f), inv2);
        w2 = __fmul_rn(__fmul_rn(g2, 0x1p64f), inv2);
    } else {
        w1 = 0.0f;
        w2 = 0.0f;
    }
}

// kappa: dt / sigma times the momentum sums' unit l/8 (see edge)
template <bool EXT>
__device__ __forceinline__ CellNew2 cell_update_pair(float2 shi, float2 slo, float2 M1, float2 M2, float2 m_old,
                                                 float2 v1_old, float2 v2_old, float2 rth, float2 ka, float2 kb,
                                                 float kappa, float qr, float dtf, float g, float dtau,
                                                 float h_dry, FF &clx, FF &cly)
{
    CellNew2 o;
    acc_add2(shi, slo, dup2(qr));
    float2 hi, lo;
    two_sum2(shi, slo, hi, lo);
    if (hi.x < 0.0f || (hi.x == 0.0f && lo.x < 0.0f)) {
        clx.add(-hi.x);
        clx.add(-lo.x);
        hi.x = 0.0f;
        lo.x = 0.0f;
    }
    if (hi.y < 0.0f || (hi.y == 0.0f && lo.y < 0.0f)) {
        cly.add(-hi.y);
        cly.add(-lo.y);
        hi.y = 0.0f;
        lo.y = 0.0f;
    }
    const float2 g1 = fma2(dup2(kappa), M1, mul2(m_old, v1_old));
    const float2 g2 = fma2(dup2(kappa), M2, mul2(m_old, v2_old));
    const float2 h = mul2(hi, rth);
    const float2 beta = mul2(dup2(dtf), fma2(ka, h, kb));
    const float2 nq = fma2(g1, g1, mul2(g2, g2));
    float2 ng;
    ng.x = nq.x >= 1.0e-36f ? fast_sqrt(nq.x) : norm2(g1.x, g2.x);
    ng.y = nq.y >= 1.0e-36f ? fast_sqrt(nq.y) : norm2(g1.y, g2.y);
    float2 ap = hi;
    if constexpr (EXT) ap = fma2(dup2(dtau), h, hi);
    const float2 rad = fma2(ap, ap, mul2(mul2(dup2(4.0f), beta), ng));
    const float2 den = add2(ap, make_float2(fast_sqrt(rad.x), fast_sqrt(rad.y)));
    const float2 inv2 = mul2(dup2(2.0f), make_float2(fast_rcp(den.x), fast_rcp(den.y)));
    float2 w1 = mul2(g1, inv2), w2 = mul2(g2, inv2);
    if (!(den.x > 1.0e-30f)) tiny_den(den.x, g1.x, g2.x, w1.x, w2.x);
    if (!(den.y > 1.0e-30f)) tiny_den(den.y, g1.y, g2.y, w1.y, w2.y);
    if constexpr (EXT) {
        if (h.x < h_dry) w1.x = w2.x = 0.0f;     // optional dry threshold (0: none)
        if (h.y < h_dry) w1.y = w2.y = 0.0f;
    }
    o.hi = hi;
    o.lo = lo;
    o.v1 = w1;
    o.v2 = w2;
    const float2 sp = fma2(w1, w1, mul2(w2, w2));
    const float2 gh = mul2(dup2(g), h);
    const float2 c = add2(make_float2(fast_sqrt(sp.x), fast_sqrt(sp.y)), make_float2(fast_sqrt(gh.x), fast_sqrt(gh.y)));
    o.cb0 = speed_bits(c.x);
    o.cb1 = speed_bits(c.y);
    return o;
}

// The common case of cell_update_pair without its branches: the same operations, hence
// the same bits, whenever no component is clamped (m < 0), has a momentum norm below
// 1e-18 or a friction denominator at or below 1e-30; rare is set when one of those (or a
// NaN) occurs, and the caller then recomputes the pair with cell_update_pair.
template <bool EXT>
__device__ __forceinline__ CellNew2 cell_update_fast(float2 shi, float2 slo, float2 M1, float2 M2, float2 m_old,
                                                 float2 v1_old, float2 v2_old, float2 rth, float2 ka, float2 kb,
                                                 float kappa, float qr, float dtf, float g, float dtau,
                                                 float h_dry, bool &rare)
{
    CellNew2 o;
    acc_add2(shi, slo, dup2(qr));
    float2 hi, lo;
    two_sum2(shi, slo, hi, lo);
    // after the renormalising two-sum hi == 0 implies lo == 0 (a float sum rounds to
    // zero only when it is zero), so a negative mass shows in hi alone
    const bool clx = hi.x < 0.0f, cly = hi.y < 0.0f;
    const float2 g1 = fma2(dup2(kappa), M1, mul2(m_old, v1_old));
    const float2 g2 = fma2(dup2(kappa), M2, mul2(m_old, v2_old));
    const float2 h = mul2(hi, rth);
    const float2 beta = mul2(dup2(dtf), fma2(ka, h, kb));
    const float2 nq = fma2(g1, g1, mul2(g2, g2));
    const float2 ng = make_float2(fast_sqrt(nq.x), fast_sqrt(nq.y));
    float2 ap = hi;
    if constexpr (EXT) ap = fma2(dup2(dtau), h, hi);
    const float2 rad = fma2(ap, ap, mul2(mul2(dup2(4.0f), beta), ng));
    const float2 den = add2(ap, make_float2(fast_sqrt(rad.x), fast_sqrt(rad.y)));
    const float2 inv2 = mul2(dup2(2.0f), make_float2(fast_rcp(den.x), fast_rcp(den.y)));
    float2 w1 = mul2(g1, inv2), w2 = mul2(g2, inv2);
    if constexpr (EXT) {
        if (h.x < h_dry) w1.x = w2.x = 0.0f;
        if (h.y < h_dry) w1.y = w2.y = 0.0f;
    }
    rare = clx || cly || !(nq.x >= 1.0e-36f) || !(nq.y >= 1.0e-36f) || !(den.x > 1.0e-30f) ||
           !(den.y > 1.0e-30f);
    o.hi = hi;
    o.lo = lo;
    o.v1 = w1;
    o.v2 = w2;
    const float2 sp = fma2(w1, w1, mul2(w2, w2));
    const float2 gh = mul2(dup2(g), h);
    const float2 c = add2(make_float2(fast_sqrt(sp.x), fast_sqrt(sp.y)), make_float2(fast_sqrt(gh.x), fast_sqrt(gh.y)));
    o.cb0 = speed_bits(c.x);
    o.cb1 = speed_bits(c.y);
    return o;
}

struct PRow {
    PCell X[2];
    float2 th[2];     // porosity theta, or in class mode the class ids' bits
    PAcc A[2];
};

// ----------------------------------------------------------------- the tile

template <bool CLS, bool EXT>
struct Tile {
    static constexpr int kHalf = kSW / 2;
    const StepArgs &a;
    StripSmem<CLS> &S;
    const float (*cls)[kMaxClasses];   // shared copies of the class tables 1/theta, a, b
    const StripMaps &maps;
    int par, np, lane, c0, r0, Hn, nchunks;
    float kappa, kl2, qr, dtf;
    unsigned cwb = 0u;
    FF outd, clq;
    bool timed_out = false;
    int n_issued = 0;

    int jown;            // first local row this tile writes
    bool own_l, own_r;   // this lane's left / right columns are written by this tile

    __device__ __forceinline__ Tile(const StepArgs &a_, StripSmem<CLS> &S_, const float (*cls_)[kMaxClasses],
                                    const StripMaps &m_, int c0_, int r0_, int own_c, int own_r_)
        : a(a_), S(S_), cls(cls_), maps(m_)
    {
        const DevCtl *ctl = a.ctl;
        par = ctl->parity;
        np = par ^ 1;
        kappa = ctl->kappa;
        qr = ctl->qr;
        dtf = ctl->dtf;
        kl2 = kappa * (0.5f * a.l);
        lane = threadIdx.x & 31;
        Hn = a.tile_rows;
        nchunks = (Hn + 2 + kRB - 1) / kRB;
        place(c0_, r0_, own_c, own_r_);
    }

    // Puts the worker on the tile at (c0_, r0_) owning columns from own_c and rows from
    // own_r_ on.  A warp that runs several tiles in one step (the strip ensemble kernel)
    // moves one worker from tile to tile: the step's reductions cwb, outd and clq carry
    // on, and the ring's barriers must have been reset in between.
    __device__ __forceinline__ void place(int c0_, int r0_, int own_c, int own_r_)
    {
        c0 = c0_;
        r0 = r0_;
        jown = 1 + (own_r_ - r0);
        own_l = c0 + 2 * lane >= own_c;
        own_r = c0 + kHalf + 2 * lane >= own_c;
        timed_out = false;
        n_issued = 0;
    }

    __device__ __forceinline__ void issue(int k)
    {
        // refuse a misaligned tensor copy (it would stop the context): flag and skip;
        // the waits then run out and the step reports ASX_ETIMEOUT
        if (((c0 - kXO) & 15) != 0 || (c0 & 3) != 0) {
            atomicOr(&a.ctl->err, kErrTimeout);
            return;
        }
        Chunk<CLS> &ch = S.ring[k % kNC];
        unsigned long long *bar = &S.bar[k % kNC];
        const int y = r0 - 1 + k * kRB;
        const unsigned bytes = (unsigned)(4 * kRB * kBXF * 4 + kRB * kSW * 4) +
                               (unsigned)(CLS ? kRB * kBXC : kRB * kBXF * 4);
        mbar_expect_tx(bar, bytes);
        tma_load_2d(&ch.mhi.v[0][0], &maps.mhi[par], c0 - kXO, y, bar);
        tma_load_2d(&ch.v1.v[0][0], &maps.v1[par], c0 - kXO, y, bar);
        tma_load_2d(&ch.v2.v[0][0], &maps.v2[par], c0 - kXO, y, bar);
        tma_load_2d(&ch.z.v[0][0], &maps.z, c0 - kXO, y, bar);
        if constexpr (CLS) tma_load_2d(&ch.th.v[0][0], &maps.th, c0 - kXOC, y, bar);
        else tma_load_2d(&ch.th.v[0][0], &maps.th, c0 - kXO, y, bar);
        tma_load_2d(&ch.mlo.v[0][0], &maps.mlo[par], c0, y, bar);
    }

    // Waits for the chunk of local row jr when jr is its first row; returns the chunk.
    __device__ __forceinline__ const Chunk<CLS> &arrive(int jr)
    {
        const int k = jr / kRB;
        if (jr % kRB == 0 && !mbar_wait_bounded(&S.bar[k % kNC], (unsigned)((k / kNC) & 1))) timed_out = true;
        return S.ring[k % kNC];
    }

    // Local row jr is done (its edges and the ones to the row below are in): once every
    // row of its chunk is, refill the chunk's slot with the chunk kNC further on.
    __device__ __forceinline__ void release(int jr)
    {
        if ((jr + 1) % kRB != 0) return;
        const int k = jr / kRB;
        __syncwarp();
        if (lane == 0 && k + kNC < nchunks) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + kNC);
            n_issued = k + kNC + 1;
        }
    }

    // The pair of ring cells at float index x and x + 64 of local row jr (the row's
    // chunk is still resident).
    __device__ __forceinline__ PCell ring_pair(int jr, int x) const
    {
        const Chunk<CLS> &ch = S.ring[(jr / kRB) % kNC];
        const int rr = jr % kRB;
        x = ASX_RING(a, x, kBXF - kHalf);
        PCell c;
        c.m = make_float2(ch.mhi.v[rr][x], ch.mhi.v[rr][x + kHalf]);
        c.v1 = make_float2(ch.v1.v[rr][x], ch.v1.v[rr][x + kHalf]);
        c.v2 = make_float2(ch.v2.v[rr][x], ch.v2.v[rr][x + kHalf]);
        c.z = make_float2(ch.z.v[rr][x], ch.z.v[rr][x + kHalf]);
        float2 rt;
        if constexpr (CLS) {
            rt = make_float2(cls[0][ch.th.v[rr][x - kXO + kXOC]], cls[0][ch.th.v[rr][x - kXO + kXOC + kHalf]]);
        } else {
            rt = make_float2(fast_rcp(ch.th.v[rr][x]), fast_rcp(ch.th.v[rr][x + kHalf]));
        }
        c.h = mul2(c.m, rt);
        return c;
    }

    // Loads local row jr (global r0 - 1 + jr) into R.
    __device__ __forceinline__ void load(int jr, PRow &R)
    {
        const int rr = jr % kRB;
        const Chunk<CLS> &ch = arrive(jr);
        const int x = ASX_RING(a, kXO + 2 * lane, kBXF - kHalf - 1), xl = ASX_RING(a, 2 * lane, kSW - kHalf - 1);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            PCell &P = R.X[e];
            P.m = make_float2(ch.mhi.v[rr][x + e], ch.mhi.v[rr][x + e + kHalf]);
            P.v1 = make_float2(ch.v1.v[rr][x + e], ch.v1.v[rr][x + e + kHalf]);
            P.v2 = make_float2(ch.v2.v[rr][x + e], ch.v2.v[rr][x + e + kHalf]);
            P.z = make_float2(ch.z.v[rr][x + e], ch.z.v[rr][x + e + kHalf]);
            float2 rt;
            if constexpr (CLS) {
                const int il = ch.th.v[rr][kXOC + xl + e], ir = ch.th.v[rr][kXOC + xl + e + kHalf];
                R.th[e] = make_float2(__int_as_float(il), __int_as_float(ir));
                rt = make_float2(cls[0][il], cls[0][ir]);
            } else {
                const float tl = ch.th.v[rr][x + e], tr = ch.th.v[rr][x + e + kHalf];
                R.th[e] = make_float2(tl, tr);
                rt = make_float2(fast_rcp(tl), fast_rcp(tr));
            }
            P.h = mul2(P.m, rt);
            R.A[e] = PAcc{P.m, make_float2(ch.mlo.v[rr][xl + e], ch.mlo.v[rr][xl + e + kHalf]), dup2(0.0f),
                          dup2(0.0f)};
        }
    }

    // Edge terms between row j (C, global row r) and row j+1 (N), and the east edges of
    // row r; ODD: parity of r.  Pair e = 0, 1 holds the columns c = c0 + 2L + e (and
    // c + 64).  Both rows always accumulate: a row this tile does not update (a halo
    // row, or a row above an overlapping last row block) is never finished, so its sums
    // are simply dropped.
    template <int ODD>
    __device__ __forceinline__ void edges(int j, PRow &C, PRow &N)
    {
        const float2 kh = dup2(0.5f * kl2);     // the scaled form's kl2 / 2
        const float vs = 8.0f / a.l;            // the momentum unit's inverse
        // the cells west and east of this lane's two, read from the ring (the same
        // values, hence the same h, as the neighbouring lanes' own cells)
        const int xw = kXO + 2 * lane - 1, xe = kXO + 2 * lane + 2;
        const PCell Wc = ring_pair(j, xw), Ec = ring_pair(j, xe);
        // ---- east edges of row r (the west edge of c_0 is the west lane's, again)
        edge<0, EXT>(a, Wc, C.X[0], kh, vs, C.A[0], false, C.A[0], true);
        edge<0, EXT>(a, C.X[0], C.X[1], kh, vs, C.A[0], true, C.A[1], true);
        edge<0, EXT>(a, C.X[1], Ec, kh, vs, C.A[1], true, C.A[1], false);
        if (ODD) {
            // odd r: NE(c) = (r+1, c+1), NW(c) = (r+1, c)
            const PCell On = ring_pair(j + 1, xe);                                // (r+1, c_1 + 1)
            edge<2, EXT>(a, C.X[0], N.X[0], kh, vs, C.A[0], true, N.A[0], true);   // NW
            edge<1, EXT>(a, C.X[0], N.X[1], kh, vs, C.A[0], true, N.A[1], true);   // NE
            edge<2, EXT>(a, C.X[1], N.X[1], kh, vs, C.A[1], true, N.A[1], true);   // NW
            edge<1, EXT>(a, C.X[1], On, kh, vs, C.A[1], true, C.A[1], false);      // NE
            // SW edge of (r+1, c_0): the NE edge of (r, c_0 - 1)
            edge<1, EXT>(a, Wc, N.X[0], kh, vs, N.A[0], false, N.A[0], true);
        } else {
            // even r: NE(c) = (r+1, c), NW(c) = (r+1, c-1)
            const PCell On = ring_pair(j + 1, xw);                                // (r+1, c_0 - 1)
            edge<1, EXT>(a, C.X[0], N.X[0], kh, vs, C.A[0], true, N.A[0], true);   // NE
            edge<2, EXT>(a, C.X[0], On, kh, vs, C.A[0], true, C.A[0], false);      // NW
            edge<1, EXT>(a, C.X[1], N.X[1], kh, vs, C.A[1], true, N.A[1], true);   // NE
            edge<2, EXT>(a, C.X[1], N.X[0], kh, vs, C.A[1], true, N.A[0], true);   // NW
            // SE edge of (r+1, c_1): the NW edge of (r, c_1 + 1)
            edge<2, EXT>(a, Ec, N.X[1], kh, vs, N.A[1], false, N.A[1], true);
        }
    }

    // Finishes the cells of row r and writes the ones this tile owns to the other state
    // buffer.
    __device__ __forceinline__ void finish(int r, PRow &C)
    {
        CellNew2 o[2];
        bool rare[2];
        const float km = kappa * (0.125f * a.l), dtau = __fmul_rn(dtf, a.tau);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            float2 rt, ka, kb;
            coeffs(C, e, rt, ka, kb);
            o[e] = cell_update_fast<EXT>(C.A[e].hi, C.A[e].lo, C.A[e].m1, C.A[e].m2, C.X[e].m, C.X[e].v1,
                                         C.X[e].v2, rt, ka, kb, km, qr, dtf, a.g, dtau, a.h_dry, rare[e]);
        }
        FF cll, clr;
        if (rare[0] || rare[1]) {
            // a clamp, a vanishing momentum or friction denominator, or a NaN: the full
            // update with its branches, for the pair(s) concerned
#pragma unroll
            for (int e = 0; e < 2; e++) {
                if (!rare[e]) continue;
                float2 rt, ka, kb;
                coeffs(C, e, rt, ka, kb);
                o[e] = cell_update_pair<EXT>(C.A[e].hi, C.A[e].lo, C.A[e].m1, C.A[e].m2, C.X[e].m, C.X[e].v1,
                                             C.X[e].v2, rt, ka, kb, km, qr, dtf, a.g, dtau, a.h_dry, cll, clr);
            }
            if (own_l && (cll.hi != 0.0f || cll.lo != 0.0f)) {
                clq.add(cll.hi);
                clq.add(cll.lo);
            }
            if (own_r && (clr.hi != 0.0f || clr.lo != 0.0f)) {
                clq.add(clr.hi);
                clq.add(clr.lo);
            }
        }
        const size_t k0 = (size_t)r * a.pitch + c0 + 2 * lane;
        if (!ASX_STORE_OK(a, (long long)k0 + kHalf + 1, (long long)a.rows * a.pitch) || !ASX_STORE_OK(a, c0 + 2 * lane + kHalf + 1, a.cols))
            return;
        if (own_l) {
            *reinterpret_cast<float2 *>(a.mhi[np] + k0) = make_float2(o[0].hi.x, o[1].hi.x);
            *reinterpret_cast<float2 *>(a.mlo[np] + k0) = make_float2(o[0].lo.x, o[1].lo.x);
            *reinterpret_cast<float2 *>(a.v1[np] + k0) = make_float2(o[0].v1.x, o[1].v1.x);
            *reinterpret_cast<float2 *>(a.v2[np] + k0) = make_float2(o[0].v2.x, o[1].v2.x);
            cwb = max(cwb, max(o[0].cb0, o[1].cb0));
        }
        if (own_r) {
            *reinterpret_cast<float2 *>(a.mhi[np] + k0 + kHalf) = make_float2(o[0].hi.y, o[1].hi.y);
            *reinterpret_cast<float2 *>(a.mlo[np] + k0 + kHalf) = make_float2(o[0].lo.y, o[1].lo.y);
            *reinterpret_cast<float2 *>(a.v1[np] + k0 + kHalf) = make_float2(o[0].v1.y, o[1].v1.y);
            *reinterpret_cast<float2 *>(a.v2[np] + k0 + kHalf) = make_float2(o[0].v2.y, o[1].v2.y);
            cwb = max(cwb, max(o[0].cb1, o[1].cb1));
        }
    }

    // Porosity terms of pair e of row C: 1/theta, alpha_p (1 - theta), theta alpha_s.
    __device__ __forceinline__ void coeffs(const PRow &C, int e, float2 &rt, float2 &ka, float2 &kb) const
    {
        if constexpr (CLS) {
            const int il = __float_as_int(C.th[e].x), ir = __float_as_int(C.th[e].y);
            rt = make_float2(cls[0][il], cls[0][ir]);
            ka = make_float2(cls[1][il], cls[1][ir]);
            kb = make_float2(cls[2][il], cls[2][ir]);
        } else {
            const float2 t = C.th[e];
            rt = make_float2(fast_rcp(t.x), fast_rcp(t.y));
            ka = mul2(dup2(a.alpha_p), sub2(dup2(1.0f), t));
            kb = mul2(t, dup2(a.alpha_s));
        }
    }

    // One row step: load row j+1, evaluate the edges of row j, finish row j, free row j's
    // ring space.
    template <int ODD>
    __device__ __forceinline__ void step_row(int j, PRow &C, PRow &N)
    {
        load(j + 1, N);
        if (j + 1 >= jown) {                // else: rows above the ones this tile writes
            edges<ODD>(j, C, N);
            if (j >= jown) finish(r0 - 1 + j, C);
        }
        release(j);
    }

    __device__ void run()
    {
        if (lane == 0) {
            for (int k = 0; k < kNC; k++) mbar_init(&S.bar[k], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int k = 0; k < kNC && k < nchunks; k++) issue(k);
            n_issued = min(kNC, nchunks);
        }
        __syncwarp();
        PRow R0, R1;
        load(0, R0);
        // local row j is global row r0 - 1 + j; every tile starts on an odd row r0, so
        // even j are even rows and one loop with two row bodies covers every tile
        for (int j = 0; j <= Hn; j += 2) {
            step_row<0>(j, R0, R1);
            if (__any_sync(0xffffffffu, timed_out) || j + 1 > Hn) return;
            step_row<1>(j + 1, R1, R0);
            if (__any_sync(0xffffffffu, timed_out)) return;
        }
    }
};

// Frame unit: kFrameCells consecutive cells of the frame, one per lane of a warp per round.
template <bool EXT>
__device__ __forceinline__ void frame_cells(const StepArgs &a, long long f0, unsigned &cwb, FF &outd,
                                            FF &clq)
{
    const StepScalars sc = step_scalars(a);
    const int ry1 = a.rye, cx1 = a.cxe;
    const int wcols = a.cx0 + (a.cols - cx1);     // frame columns of the interior rows
    for (int i = (int)(threadIdx.x & 31); i < kFrameCells; i += 32) {
        const long long f = f0 + i;
        if (f >= a.frame_n) break;
        int r, c;
        if (f < a.frame_a) {
            const int ra = (int)(f / a.cols);
            r = ra < a.ry0 ? ra : ry1 + (ra - a.ry0);
            c = (int)(f - (long long)ra * a.cols);
        } else {
            const long long g = f - a.frame_a;
            const int rb = (int)(g / wcols), cb = (int)(g - (long long)rb * wcols);
            r = a.ry0 + rb;
            c = cb < a.cx0 ? cb : cx1 + (cb - a.cx0);
        }
        gather_cell<EXT>(a, sc, r, c, cwb, outd, clq);
    }
}

}  // namespace
}  // namespace asx
