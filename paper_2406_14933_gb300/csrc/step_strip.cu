// step_strip.cu -- the main step kernel: one warp marches down a 128-column tile fed by
// TMA, four cells per lane.
//
// Same arithmetic as the gather kernel (Sec. 2.2, Eq. fvm_2D_eq_frac.07 in the form of
// Appendix A), organised for GB300:
//   * a CTA is one warp and owns kSW = 128 columns x H rows; lane L owns the four
//     adjacent cells at columns c0 + 4L .. c0 + 4L + 3;
//   * rows r0-1 .. r0+H of every field (one halo row above and below, halo columns left
//     and right) stream into a shared-memory ring of 2-row chunks through TMA tensor
//     loads (cp.async.bulk.tensor.2d) that complete on mbarriers; lane 0 refills a chunk
//     once every row of it is finished;
//   * the warp walks the tile row by row; the edges between row r and r+1 and the east
//     edges of row r are evaluated by the lane that owns their lower cell; a lane also
//     evaluates the one horizontal and one diagonal edge it shares with each neighbouring
//     lane (the same canonical edge, so the same bits), which replaces every exchange of
//     edge terms; every lane reads the cells beside its four (in its own row and the
//     next, including the halo columns at the tile ends) from the ring: the same values,
//     hence the same bits, as the neighbouring lane's own cells;
//   * contributions to row r+1 stay in registers until that row is finished; no block
//     barrier is needed;
//   * tiles are laid out so that each tile with its halo lies inside the raster, which
//     leaves no boundary edge in the tile code; the remaining cells along the raster
//     sides (the frame) are processed in the same launch by frame CTAs that gather each
//     cell's six neighbours (the same per-cell code as the gather kernel).
// Both cells of an edge accumulate the mass increment of the same canonical edge
// function, so opposite increments are bit-identical and the water budget closes to
// float64 rounding.
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

// ----------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
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

// Bounded wait on an mbarrier phase: gives up after ~2^26 polls (well over a second).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    for (unsigned it = 0; it < (1u << 26); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

// ----------------------------------------------------------------- cell helpers

struct Acc {
    float hi, lo, m1, m2;    // compensated mass, momentum sums J + S
};

// Edge (X lower, Y upper) in direction D; adds its terms to ax if ux and to ay if uy
// (a side not used belongs to another lane or is not updated by this tile).
// The pressure term p = c dh enters each momentum sum through one fused multiply-add.
// EXT: the optional terms are compiled in; with a.visc the artificial viscosity adds
// t (v_Y - v_X) to X and t (v_X - v_Y) to Y.
template <int D, bool EXT>
__device__ __forceinline__ void edge(const StepArgs &a, const Cell &X, const Cell &Y, float kl2,
                                     Acc &ax, bool ux, Acc &ay, bool uy)
{
    float q, f1, f2, dh;
    edge_core<D>(X, Y, kl2, 0.25f * a.l, q, f1, f2, dh);
    const float c1 = a.cpe[D][0], c2 = a.cpe[D][1];
    if (ux) {
        acc_add(ax.hi, ax.lo, -q);
        ax.m1 = __fsub_rn(__fmaf_rn(c1, dh, ax.m1), f1);
        ax.m2 = __fsub_rn(__fmaf_rn(c2, dh, ax.m2), f2);
    }
    if (uy) {
        acc_add(ay.hi, ay.lo, q);
        ay.m1 = __fadd_rn(__fmaf_rn(c1, dh, ay.m1), f1);
        ay.m2 = __fadd_rn(__fmaf_rn(c2, dh, ay.m2), f2);
    }
    if (EXT && a.visc) {
        const float t = visc_coef(X, Y, a.l, a.g);
        const float d1 = __fsub_rn(Y.v1, X.v1), d2 = __fsub_rn(Y.v2, X.v2);
        if (ux) {
            ax.m1 = __fmaf_rn(t, d1, ax.m1);
            ax.m2 = __fmaf_rn(t, d2, ax.m2);
        }
        if (uy) {
            ay.m1 = __fmaf_rn(-t, d1, ay.m1);
            ay.m2 = __fmaf_rn(-t, d2, ay.m2);
        }
    }
}

// Per-lane state of one row: four cells, their porosity (theta, or in class mode the
// class id's bits) and the accumulators of their edge terms.  The halo cells at both ends
// of the tile row are read from the ring when needed.
struct Row {
    Cell X[4];
    float th[4];
    Acc A[4];
};

// ----------------------------------------------------------------- the tile

template <bool CLS, bool EXT>
struct Tile {
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

    int jown;          // first local row this tile writes
    bool lane_own;     // this lane's four columns are written by this tile

    __device__ __forceinline__ Tile(const StepArgs &a_, StripSmem<CLS> &S_, const float (*cls_)[kMaxClasses],
                                    const StripMaps &m_, int c0_, int r0_, int own_c, int own_r)
        : a(a_), S(S_), cls(cls_), maps(m_)
    {
        const DevCtl *ctl = a.ctl;
        par = ctl->parity;
        np = par ^ 1;
        kappa = ctl->kappa;
        qr = ctl->qr;
        dtf = ctl->dtf;
        kl2 = kappa * (0.5f * a.l);
        lane = threadIdx.x;
        c0 = c0_;
        r0 = r0_;
        Hn = a.tile_rows;
        jown = 1 + (own_r - r0);
        lane_own = c0 + 4 * lane >= own_c;
        nchunks = (Hn + 2 + kRB - 1) / kRB;
    }

    __device__ __forceinline__ int col(int e) const { return c0 + 4 * lane + e; }

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

    // Halo cell of ring row rr at float index x.
    __device__ __forceinline__ Cell ring_cell(const Chunk<CLS> &ch, int rr, int x) const
    {
        Cell c;
        c.m = ch.mhi.v[rr][x];
        c.v1 = ch.v1.v[rr][x];
        c.v2 = ch.v2.v[rr][x];
        c.z = ch.z.v[rr][x];
        float rt;
        if constexpr (CLS) rt = cls[0][ch.th.v[rr][x - kXO + kXOC]];
        else rt = fast_rcp(ch.th.v[rr][x]);
        c.h = __fmul_rn(c.m, rt);
        return c;
    }

    // The cell of local row jr at ring x index x (the row's chunk is still resident).
    __device__ __forceinline__ Cell ring_at(int jr, int x) const
    {
        return ring_cell(S.ring[(jr / kRB) % kNC], jr % kRB, x);
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

    // Loads local row jr (global r0 - 1 + jr) into R.
    __device__ __forceinline__ void load(int jr, Row &R)
    {
        const int k = jr / kRB, rr = jr % kRB;
        if (rr == 0 && !mbar_wait_bounded(&S.bar[k % kNC], (unsigned)((k / kNC) & 1))) timed_out = true;
        const Chunk<CLS> &ch = S.ring[k % kNC];
        const int x = kXO + 4 * lane;
        const float4 m4 = *reinterpret_cast<const float4 *>(&ch.mhi.v[rr][x]);
        const float4 u4 = *reinterpret_cast<const float4 *>(&ch.v1.v[rr][x]);
        const float4 w4 = *reinterpret_cast<const float4 *>(&ch.v2.v[rr][x]);
        const float4 z4 = *reinterpret_cast<const float4 *>(&ch.z.v[rr][x]);
        const float4 l4 = *reinterpret_cast<const float4 *>(&ch.mlo.v[rr][4 * lane]);
        const float mm[4] = {m4.x, m4.y, m4.z, m4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w};
        const float ww[4] = {w4.x, w4.y, w4.z, w4.w}, zz[4] = {z4.x, z4.y, z4.z, z4.w};
        const float ll[4] = {l4.x, l4.y, l4.z, l4.w};
        if constexpr (CLS) {
            const uchar4 c4 = *reinterpret_cast<const uchar4 *>(&ch.th.v[rr][kXOC + 4 * lane]);
            const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                R.th[e] = __int_as_float(cc[e]);
                R.X[e].h = __fmul_rn(mm[e], cls[0][cc[e]]);
            }
        } else {
            const float4 t4 = *reinterpret_cast<const float4 *>(&ch.th.v[rr][x]);
            const float tt[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                R.th[e] = tt[e];
                R.X[e].h = __fmul_rn(mm[e], fast_rcp(tt[e]));
            }
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
            R.X[e].m = mm[e];
            R.X[e].v1 = uu[e];
            R.X[e].v2 = ww[e];
            R.X[e].z = zz[e];
            R.A[e] = Acc{mm[e], ll[e], 0.0f, 0.0f};
        }
    }

    // Edge terms between row j (C, global row r) and row j+1 (N), and the east edges of
    // row r; ODD: parity of r.  Both rows always accumulate: a row this tile does not
    // update (a halo row, or a row above an overlapping last row block) is never
    // finished, so its sums are simply dropped.
    template <int ODD>
    __device__ __forceinline__ void edges(int j, Row &C, Row &N)
    {
        // the cells west and east of this lane's four, read from the ring (the same
        // values, hence the same h, as the neighbouring lane's own cells)
        const int xw = kXO + 4 * lane - 1, xe = kXO + 4 * lane + 4;
        const Cell Wc = ring_at(j, xw);
        const Cell Ec = ring_at(j, xe);
        // ---- east edges of row r (the west edge of c_0 is the west lane's, again)
        edge<0, EXT>(a, Wc, C.X[0], kl2, C.A[0], false, C.A[0], true);
#pragma unroll
        for (int e = 0; e < 3; e++) edge<0, EXT>(a, C.X[e], C.X[e + 1], kl2, C.A[e], true, C.A[e + 1], true);
        edge<0, EXT>(a, C.X[3], Ec, kl2, C.A[3], true, C.A[3], false);
        if (ODD) {
            // odd r: NE(c) = (r+1, c+1), NW(c) = (r+1, c)
            const Cell On = ring_at(j + 1, xe);                                   // (r+1, c_3 + 1)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                edge<2, EXT>(a, C.X[e], N.X[e], kl2, C.A[e], true, N.A[e], true);        // NW
                if (e < 3) edge<1, EXT>(a, C.X[e], N.X[e + 1], kl2, C.A[e], true, N.A[e + 1], true);
                else edge<1, EXT>(a, C.X[3], On, kl2, C.A[3], true, C.A[3], false);
            }
            // SW edge of (r+1, c_0): the NE edge of (r, c_0 - 1)
            edge<1, EXT>(a, Wc, N.X[0], kl2, N.A[0], false, N.A[0], true);
        } else {
            // even r: NE(c) = (r+1, c), NW(c) = (r+1, c-1)
            const Cell On = ring_at(j + 1, xw);                                   // (r+1, c_0 - 1)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                edge<1, EXT>(a, C.X[e], N.X[e], kl2, C.A[e], true, N.A[e], true);        // NE
                if (e >= 1) edge<2, EXT>(a, C.X[e], N.X[e - 1], kl2, C.A[e], true, N.A[e - 1], true);
                else edge<2, EXT>(a, C.X[0], On, kl2, C.A[0], true, C.A[0], false);
            }
            // SE edge of (r+1, c_3): the NW edge of (r, c_3 + 1)
            edge<2, EXT>(a, Ec, N.X[3], kl2, N.A[3], false, N.A[3], true);
        }
    }

    // Finishes the cells of row r and writes them to the other state buffer.
    __device__ __forceinline__ void finish(int r, Row &C)
    {
        CellNew o[4];
        FF cl;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            float rt, ka, kb;
            if constexpr (CLS) {
                const int k = __float_as_int(C.th[e]);
                rt = cls[0][k];
                ka = cls[1][k];
                kb = cls[2][k];
            } else {
                const float t = C.th[e];
                rt = fast_rcp(t);
                ka = a.alpha_p * (1.0f - t);
                kb = t * a.alpha_s;
            }
            o[e] = cell_update<EXT>(C.A[e].hi, C.A[e].lo, C.A[e].m1, C.A[e].m2, C.X[e].m, C.X[e].v1, C.X[e].v2,
                               rt, ka, kb, kappa, qr, dtf, a.g, __fmul_rn(dtf, a.tau), a.h_dry, cl);
        }
        if (!lane_own) return;       // columns written by the neighbouring tile
        if (cl.hi != 0.0f || cl.lo != 0.0f) {
            clq.add(cl.hi);
            clq.add(cl.lo);
        }
        const size_t k0 = (size_t)r * a.pitch + col(0);
        *reinterpret_cast<float4 *>(a.mhi[np] + k0) = make_float4(o[0].hi, o[1].hi, o[2].hi, o[3].hi);
        *reinterpret_cast<float4 *>(a.mlo[np] + k0) = make_float4(o[0].lo, o[1].lo, o[2].lo, o[3].lo);
        *reinterpret_cast<float4 *>(a.v1[np] + k0) = make_float4(o[0].v1, o[1].v1, o[2].v1, o[3].v1);
        *reinterpret_cast<float4 *>(a.v2[np] + k0) = make_float4(o[0].v2, o[1].v2, o[2].v2, o[3].v2);
#pragma unroll
        for (int e = 0; e < 4; e++) cwb = max(cwb, o[e].cbits);
    }

    // One row step: load row j+1, evaluate the edges of row j, finish row j, free row j's
    // ring space.
    template <int ODD>
    __device__ __forceinline__ void step_row(int j, Row &C, Row &N)
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
        Row R0, R1;
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

// Frame CTA: kFrameCells consecutive cells of the frame, one per lane per round.
template <bool EXT>
__device__ __forceinline__ void frame_cells(const StepArgs &a, long long f0, unsigned &cwb, FF &outd,
                                            FF &clq)
{
    const StepScalars sc = step_scalars(a);
    const int ry1 = a.rye, cx1 = a.cxe;
    const int wcols = a.cx0 + (a.cols - cx1);     // frame columns of the interior rows
    for (int i = threadIdx.x; i < kFrameCells; i += 32) {
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

// 128 registers and a 2 x 2-row ring (13.6 KB) let 15-16 one-warp CTAs share an SM
template <bool CLS, bool EXT>
__global__ void __launch_bounds__(32, ASX_STRIP_MINB) step_strip_kernel(const StepArgs a, const __grid_constant__ StripMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment: align the dynamic block by hand
    StripSmem<CLS> &S = *reinterpret_cast<StripSmem<CLS> *>(
        smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    if (!a.ctl->active) return;
    // class tables, indexed per cell: from the parameter space into shared memory
    __shared__ float s_cls[3][kMaxClasses];
    if (CLS && threadIdx.x < kMaxClasses) {
        s_cls[0][threadIdx.x] = a.cls_rth[threadIdx.x];
        s_cls[1][threadIdx.x] = a.cls_a[threadIdx.x];
        s_cls[2][threadIdx.x] = a.cls_b[threadIdx.x];
    }
    __syncwarp();
    unsigned cwb = 0u;
    double outq = 0.0, clq = 0.0;
    if ((int)blockIdx.x < a.ntiles) {
        const int ns = a.nstrips + (a.cx_last >= 0 ? 1 : 0);
        const int strip = blockIdx.x % ns, rblk = blockIdx.x / ns;
        const int c0 = strip < a.nstrips ? a.cx0 + strip * kSW : a.cx_last;
        const int own_c = strip < a.nstrips ? c0 : a.cx0 + a.nstrips * kSW;
        const int r0 = rblk < a.nrb ? a.ry0 + rblk * a.tile_rows : a.r_last;
        const int own_r = rblk < a.nrb ? r0 : a.ry0 + a.nrb * a.tile_rows;
        if ((r0 & 1) == 0) {
            // the layout puts every tile on an odd first row; anything else is refused
            // before a copy is issued
            if (threadIdx.x == 0) atomicOr(&a.ctl->err, kErrTimeout);
            return;
        }
        Tile<CLS, EXT> T(a, S, s_cls, maps, c0, r0, own_c, own_r);
        T.run();
        if (__any_sync(0xffffffffu, T.timed_out)) {
            // a tensor copy did not arrive in time: flag the error, wait (bounded) for
            // the copies still in flight, and leave without finishing the step
            if (threadIdx.x == 0) {
                atomicOr(&a.ctl->err, kErrTimeout);
                for (int k = max(0, T.n_issued - kNC); k < T.n_issued; k++)
                    mbar_wait_bounded(&S.bar[k % kNC], (unsigned)((k / kNC) & 1));
            }
            return;
        }
        cwb = T.cwb;
        outq = T.outd.value();
        clq = T.clq.value();
    } else {
        FF o, cl;
        frame_cells<EXT>(a, (long long)(blockIdx.x - a.ntiles) * kFrameCells, cwb, o, cl);
        outq = o.value();
        clq = cl.value();
    }
    reduce_and_finish<32>(a, cwb, outq, clq);
}

}  // namespace

template <bool CLS>
size_t strip_smem() { return sizeof(StripSmem<CLS>) + 128; }

void step_strip_layout(StepArgs &a)
{
    // tiles hold an even number of rows and start on odd rows (row 1, 1 + H, ...), so
    // that every tile's first local row has the same parity
    a.tile_rows += a.tile_rows & 1;
    const int H = a.tile_rows;
    // tiles start at column 4 (TMA boxes start 4 columns to the left, on a 16-byte
    // boundary) and row 1, and their halo must end inside the raster
    a.cx0 = 4;
    a.nstrips = a.cols - 1 - a.cx0 >= kSW ? (a.cols - 1 - a.cx0) / kSW : 0;
    a.ry0 = 1;
    a.nrb = a.rows - 2 >= H ? (a.rows - 2) / H : 0;
    if (a.nstrips == 0 || a.nrb == 0) a.nstrips = a.nrb = 0;
    const int cx1 = a.cx0 + a.nstrips * kSW, ry1 = a.ry0 + a.nrb * H;
    a.cx_last = -1;
    a.cxe = cx1;
    a.r_last = -1;
    a.rye = ry1;
    if (a.nstrips > 0) {
        // last strip flush with the east side: start 4 mod 16, halo column inside
        const int cl = ((a.cols - 1 - kSW - 4) / 16) * 16 + 4;
        if (cl + kSW > cx1 && cl >= a.cx0) {
            a.cx_last = cl;
            a.cxe = cl + kSW;
        }
        int rl = a.rows - 1 - H;
        rl -= 1 - (rl & 1);                // odd first row (the frame takes a row left over)
        if (rl + H > ry1 && rl >= a.ry0) {
            a.r_last = rl;
            a.rye = rl + H;
        }
    }
    a.ntiles = (a.nstrips + (a.cx_last >= 0 ? 1 : 0)) * (a.nrb + (a.r_last >= 0 ? 1 : 0));
    if (a.nstrips == 0) a.ntiles = 0;
    const long long n = (long long)a.rows * a.cols;
    const long long inner = (long long)(a.rye - a.ry0) * (a.cxe - a.cx0);
    a.frame_n = a.ntiles ? n - inner : n;
    a.frame_a = a.ntiles ? (long long)(a.rows - (a.rye - a.ry0)) * a.cols : n;
    a.nblocks = a.ntiles + (int)((a.frame_n + kFrameCells - 1) / kFrameCells);
}

cudaError_t step_strip_configure()
{
    cudaError_t e = cudaFuncSetAttribute(step_strip_kernel<false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)strip_smem<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_strip_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)strip_smem<true>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_strip_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)strip_smem<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_strip_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)strip_smem<true>());
    return e;
}

cudaError_t launch_step_strip(const StepArgs &a, const StripMaps &maps, cudaStream_t s)
{
    // land-cover classes (uint8 ids and per-class tables) or per-cell theta; with the
    // optional terms (viscosity, linear resistance, dry threshold) or the plain scheme
    const bool ext = a.visc || a.tau > 0.0f || a.h_dry > 0.0f;
    if (a.cls) {
        if (ext) step_strip_kernel<true, true><<<a.nblocks, 32, strip_smem<true>(), s>>>(a, maps);
        else step_strip_kernel<true, false><<<a.nblocks, 32, strip_smem<true>(), s>>>(a, maps);
    } else {
        if (ext) step_strip_kernel<false, true><<<a.nblocks, 32, strip_smem<false>(), s>>>(a, maps);
        else step_strip_kernel<false, false><<<a.nblocks, 32, strip_smem<false>(), s>>>(a, maps);
    }
    return cudaGetLastError();
}

}  // namespace asx
