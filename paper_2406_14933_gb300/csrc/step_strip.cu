// step_strip.cu -- the main step kernel: TMA-fed row marching over 128-column strips.
//
// Same arithmetic as the gather kernel (Sec. 2.2, Eq. fvm_2D_eq_frac.07 in the form of
// Appendix A), organised for GB300:
//   * a CTA owns a tile of kStripW = 128 columns x H rows; 64 threads, two adjacent
//     cells each;
//   * the fields of rows r0-1 .. r0+H (one halo row above and below, four halo columns
//     left and right) stream into a shared-memory ring of 2-row chunks with TMA tensor
//     loads (cp.async.bulk.tensor.2d) completing on mbarriers; one thread refills a chunk
//     as soon as every thread has finished with it;
//   * the CTA marches down the tile one row per iteration; each edge is evaluated once,
//     by the thread that owns its lower cell (E, NE, NW edges), and the terms destined for
//     a cell of another thread are passed through shared memory; the depth h = m / theta
//     of each row is computed once and shared the same way;
//   * contributions to the row below are held in registers until that row is finished.
// The mass increment of an edge is bit-identical to the gather kernel's (same canonical
// edge function), so the water budget closes the same way.
#include <cuda.h>

#include "device_common.cuh"

namespace asx {

namespace {

constexpr int kSW = kStripW;           // tile width in cells
constexpr int kST = kSW / 2;           // threads per CTA (two cells each)
constexpr int kRB = 2;                 // rows per ring chunk
constexpr int kNC = 3;                 // chunks in the ring
constexpr int kBXF = kSW + 8;          // float box width (from column c0 - 4)
constexpr int kBXC = kSW + 32;         // uint8 box width (from column c0 - 16)
constexpr int kXO = 4;                 // ring x index of column c0 (float fields)
constexpr int kXOC = 16;               // ring x index of column c0 (class field)

struct __align__(128) FBox { float v[kRB][kBXF]; float pad[(1152 - kRB * kBXF * 4) / 4]; };
struct __align__(128) LBox { float v[kRB][kSW]; };
struct __align__(128) Chunk {
    FBox mhi, v1, v2, z, th;           // th: theta (float) or, reinterpreted, class ids
    LBox mlo;
};
static_assert(sizeof(FBox) == 1152, "box padding");
static_assert(kRB * kBXC <= (int)sizeof(FBox), "class box fits the theta slot");

struct StripSmem {
    Chunk ring[kNC];
    float hrow[2][kBXF];               // depth of the rows j and j+1 (ring x indexing)
    float eEq[kST], eE1[kST], eE2[kST];    // east edge terms for the next thread's cell a
    float eDq[kST], eD1[kST], eD2[kST];    // diagonal edge terms for a neighbour thread
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

// ----------------------------------------------------------------- the kernel

struct Acc {
    float hi, lo, m1, m2;    // compensated mass, momentum sums J + S
};

__device__ __forceinline__ void acc_in(Acc &A, float q, float u1, float u2)
{
    acc_add(A.hi, A.lo, q);
    A.m1 += u1;
    A.m2 += u2;
}

// Free-discharge contribution of a boundary edge of cell X in direction d (walls: none).
__device__ __forceinline__ void bnd(const StepArgs &a, const Cell &X, int d, int side, int pos,
                                    float kl2, Acc &A, FF &outd)
{
    if (side_is_free(a, side, pos)) free_edge(X, d, kl2, 0.5f * a.l, A.hi, A.lo, A.m1, A.m2, outd);
}

// Applies an interior edge (A lower, B upper) computed in direction D: the lower cell's
// accumulator gets -q, P - F v; the upper's (returned) terms are q, P + F v.
template <int D>
__device__ __forceinline__ void edge(const StepArgs &a, const Cell &A, const Cell &B, float kl2,
                                     Acc *accA, float &q, float &u1, float &u2)
{
    float f1, f2, p1, p2;
    edge_terms<D>(A, B, kl2, 0.25f * a.l, a.cpe[D][0], a.cpe[D][1], q, f1, f2, p1, p2);
    if (accA) acc_in(*accA, -q, p1 - f1, p2 - f2);
    u1 = p1 + f1;
    u2 = p2 + f2;
}

__device__ __forceinline__ Cell ring_cell(const Chunk &ch, int rr, int x, const float *hrow)
{
    Cell c;
    c.m = ch.mhi.v[rr][x];
    c.v1 = ch.v1.v[rr][x];
    c.v2 = ch.v2.v[rr][x];
    c.z = ch.z.v[rr][x];
    c.h = hrow[x];
    return c;
}

// 1 / theta of the ring cell at float index x (same value as cell_rtheta).
__device__ __forceinline__ float ring_rtheta(const StepArgs &a, const Chunk &ch, int rr, int x)
{
    if (a.cls) {
        const uint8_t *cl = reinterpret_cast<const uint8_t *>(&ch.th.v[0][0]);
        return a.cls_rth[cl[rr * kBXC + (x - kXO + kXOC)]];
    }
    return fast_rcp(ch.th.v[rr][x]);
}

// One tile.  IN = the tile and its halo lie inside the raster (no boundary edge, every
// cell valid): the boundary branches compile away.
template <bool IN>
__device__ __forceinline__ void strip_tile(const StepArgs &a, const StripMaps &maps, StripSmem &S,
                                           int strip, int rblk)
{
    const DevCtl *ctl = a.ctl;
    const int par = ctl->parity, np = par ^ 1;
    const float kappa = ctl->kappa, qr = ctl->qr, dtf = ctl->dtf;
    const float kl2 = kappa * (0.5f * a.l);
    const int t = threadIdx.x;
    const int H = a.tile_rows;
    const int c0 = strip * kSW, r0 = rblk * H;
    const int Hn = min(H, a.rows - r0);          // owned rows inside the raster
    const int nrows = Hn + 2;                     // local rows 0 .. Hn+1
    const int nchunks = (nrows + kRB - 1) / kRB;
    const CUtensorMap *mp_mhi = &maps.mhi[par], *mp_v1 = &maps.v1[par], *mp_v2 = &maps.v2[par];
    const CUtensorMap *mp_mlo = &maps.mlo[par];
    const unsigned chunk_bytes = (unsigned)(4 * kRB * kBXF * 4 + kRB * kSW * 4) +
                                 (unsigned)(a.cls ? kRB * kBXC : kRB * kBXF * 4);

    auto issue = [&](int k) {
        Chunk &ch = S.ring[k % kNC];
        unsigned long long *bar = &S.bar[k % kNC];
        const int y = r0 - 1 + k * kRB;
        mbar_expect_tx(bar, chunk_bytes);
        tma_load_2d(&ch.mhi.v[0][0], mp_mhi, c0 - kXO, y, bar);
        tma_load_2d(&ch.v1.v[0][0], mp_v1, c0 - kXO, y, bar);
        tma_load_2d(&ch.v2.v[0][0], mp_v2, c0 - kXO, y, bar);
        tma_load_2d(&ch.z.v[0][0], &maps.z, c0 - kXO, y, bar);
        if (a.cls) tma_load_2d(&ch.th.v[0][0], &maps.th, c0 - kXOC, y, bar);
        else tma_load_2d(&ch.th.v[0][0], &maps.th, c0 - kXO, y, bar);
        tma_load_2d(&ch.mlo.v[0][0], mp_mlo, c0, y, bar);
    };

    int n_issued = 0;                  // chunks issued (thread 0)
    if (t == 0) {
        for (int k = 0; k < kNC; k++) mbar_init(&S.bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < kNC && k < nchunks; k++) issue(k);
        n_issued = min(kNC, nchunks);
    }
    __syncthreads();

    const int ca = c0 + 2 * t, cb = ca + 1;
    const bool va = IN || ca < a.cols, vb = IN || cb < a.cols;
    const bool hasE = IN || cb + 1 < a.cols;      // b's east neighbour (r, cb+1) exists
    const bool hasW = IN || ca > 0;               // a's west neighbour (r, ca-1) exists
    const int xa = kXO + 2 * t, xb = xa + 1;

    Cell A0{}, B0{}, A1{}, B1{};     // row j (cur) and row j+1 (nxt) cells a, b
    float rtA0 = 1.f, rtB0 = 1.f, rtA1 = 1.f, rtB1 = 1.f;       // 1 / theta
    float kaA0 = 0.f, kaB0 = 0.f, kaA1 = 0.f, kaB1 = 0.f;       // alpha_p (1 - theta)
    float kbA0 = 0.f, kbB0 = 0.f, kbA1 = 0.f, kbB1 = 0.f;       // theta alpha_s
    Acc cA{}, cB{}, nA{}, nB{};      // accumulators of row j and row j+1
    unsigned cwb = 0u;               // max wave speed as float bits (NaN sorts above +Inf)
    FF outd, clq;                    // boundary outflow and clamped water of this thread
    bool timed_out = false;

    // Loads local row jr (global r0 - 1 + jr) into (A1, B1), computes its depth into
    // hrow[jr & 1] (halo columns by the edge threads) and starts its accumulators.
    auto load_row = [&](int jr) {
        const int k = jr / kRB, rr = jr % kRB;
        if (rr == 0 || jr == 0) {
            if (!mbar_wait_bounded(&S.bar[k % kNC], (unsigned)((k / kNC) & 1))) timed_out = true;
        }
        const Chunk &ch = S.ring[k % kNC];
        const int rg = r0 - 1 + jr;
        const bool in = rg >= 0 && rg < a.rows;
        float *hr = S.hrow[jr & 1];
        const float2 m2 = *reinterpret_cast<const float2 *>(&ch.mhi.v[rr][xa]);
        const float2 u2 = *reinterpret_cast<const float2 *>(&ch.v1.v[rr][xa]);
        const float2 w2 = *reinterpret_cast<const float2 *>(&ch.v2.v[rr][xa]);
        const float2 z2 = *reinterpret_cast<const float2 *>(&ch.z.v[rr][xa]);
        A1.m = m2.x; B1.m = m2.y;
        A1.v1 = u2.x; B1.v1 = u2.y;
        A1.v2 = w2.x; B1.v2 = w2.y;
        A1.z = z2.x; B1.z = z2.y;
        if (a.cls) {
            const uint8_t *cl = reinterpret_cast<const uint8_t *>(&ch.th.v[0][0]) + rr * kBXC + kXOC + 2 * t;
            const int ia = cl[0], ib = cl[1];
            rtA1 = a.cls_rth[ia]; kaA1 = a.cls_a[ia]; kbA1 = a.cls_b[ia];
            rtB1 = a.cls_rth[ib]; kaB1 = a.cls_a[ib]; kbB1 = a.cls_b[ib];
        } else {
            const float2 th2 = *reinterpret_cast<const float2 *>(&ch.th.v[rr][xa]);
            rtA1 = fast_rcp(th2.x); kaA1 = a.alpha_p * (1.0f - th2.x); kbA1 = th2.x * a.alpha_s;
            rtB1 = fast_rcp(th2.y); kaB1 = a.alpha_p * (1.0f - th2.y); kbB1 = th2.y * a.alpha_s;
        }
        A1.h = (IN || (in && va)) ? __fmul_rn(A1.m, rtA1) : 0.0f;
        B1.h = (IN || (in && vb)) ? __fmul_rn(B1.m, rtB1) : 0.0f;
        *reinterpret_cast<float2 *>(&hr[xa]) = make_float2(A1.h, B1.h);
        if (t == 0) {
            const int x = kXO - 1;
            hr[x] = (IN || (in && c0 > 0)) ? __fmul_rn(ch.mhi.v[rr][x], ring_rtheta(a, ch, rr, x)) : 0.0f;
        }
        if (t == kST - 1) {
            const int x = kXO + kSW;
            hr[x] = (IN || (in && c0 + kSW < a.cols)) ? __fmul_rn(ch.mhi.v[rr][x], ring_rtheta(a, ch, rr, x)) : 0.0f;
        }
        const float2 lo2 = *reinterpret_cast<const float2 *>(&ch.mlo.v[rr][2 * t]);
        nA = Acc{A1.m, lo2.x, 0.0f, 0.0f};
        nB = Acc{B1.m, lo2.y, 0.0f, 0.0f};
    };

    load_row(0);
    for (int j = 0; j <= Hn; j++) {
        // rotate: row j becomes current
        A0 = A1; B0 = B1;
        rtA0 = rtA1; rtB0 = rtB1; kaA0 = kaA1; kaB0 = kaB1; kbA0 = kbA1; kbB0 = kbB1;
        cA = nA; cB = nB;
        load_row(j + 1);
        if (__syncthreads_or(timed_out)) break;                    // S1
        // refill the chunk every thread has finished with (rows j-2, j-1)
        if (t == 0 && j >= 2 && (j % kRB) == 0) {
            const int kd = j / kRB - 1;
            if (kd + kNC < nchunks) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(kd + kNC);
                n_issued = kd + kNC + 1;
            }
        }
        const int r = r0 - 1 + j;
        const bool in_r = IN || (r >= 0 && r < a.rows);
        const bool in_n = IN || (r + 1 >= 0 && r + 1 < a.rows);
        const bool own = j >= 1 && in_r;
        const bool nown = j + 1 <= Hn && in_n;
        const int odd = r & 1;
        const int kc = j / kRB, rc = j % kRB, kn = (j + 1) / kRB, rn = (j + 1) % kRB;
        const Chunk &chc = S.ring[kc % kNC];
        const Chunk &chn = S.ring[kn % kNC];
        const float *hc = S.hrow[j & 1], *hn = S.hrow[(j + 1) & 1];
        float pq = 0.f, p1 = 0.f, p2 = 0.f;       // published diagonal terms
        float q, u1, u2;

        if (own) {
            // ---- horizontal edges of row r
            if (va) {
                if (vb) {
                    edge<0>(a, A0, B0, kl2, &cA, q, u1, u2);
                    acc_in(cB, q, u1, u2);
                } else {
                    bnd(a, A0, 0, ASX_SIDE_E, r, kl2, cA, outd);
                }
            }
            if (vb) {
                if (hasE) {
                    const Cell E = ring_cell(chc, rc, xb + 1, hc);
                    edge<0>(a, B0, E, kl2, &cB, q, u1, u2);
                    S.eEq[t] = q; S.eE1[t] = u1; S.eE2[t] = u2;
                } else {
                    bnd(a, B0, 0, ASX_SIDE_E, r, kl2, cB, outd);
                }
            }
            if (va) {
                if (!hasW) {
                    bnd(a, A0, 3, ASX_SIDE_W, r, kl2, cA, outd);
                } else if (t == 0) {
                    const Cell Wc = ring_cell(chc, rc, xa - 1, hc);
                    edge<0>(a, Wc, A0, kl2, nullptr, q, u1, u2);
                    acc_in(cA, q, u1, u2);
                }
            }
        }
        if (own || nown) {
            if (!IN && !in_r) {
                // row r is above the raster: the lower edges of row r+1 lie on the S side
                if (nown) {
                    if (va) { bnd(a, A1, 4, ASX_SIDE_S, ca, kl2, nA, outd); bnd(a, A1, 5, ASX_SIDE_S, ca, kl2, nA, outd); }
                    if (vb) { bnd(a, B1, 4, ASX_SIDE_S, cb, kl2, nB, outd); bnd(a, B1, 5, ASX_SIDE_S, cb, kl2, nB, outd); }
                }
            } else if (!IN && !in_n) {
                // row r+1 is beyond the raster: the upper edges of row r lie on the N side
                if (own) {
                    if (va) { bnd(a, A0, 1, ASX_SIDE_N, ca, kl2, cA, outd); bnd(a, A0, 2, ASX_SIDE_N, ca, kl2, cA, outd); }
                    if (vb) { bnd(a, B0, 1, ASX_SIDE_N, cb, kl2, cB, outd); bnd(a, B0, 2, ASX_SIDE_N, cb, kl2, cB, outd); }
                }
            } else if (!odd) {
                // even r: NE(c) = (r+1, c), NW(c) = (r+1, c-1)
                Acc *oA = own ? &cA : nullptr, *oB = own ? &cB : nullptr;
                if (va) {
                    edge<1>(a, A0, A1, kl2, oA, q, u1, u2);             // a -> nxt a
                    if (nown) acc_in(nA, q, u1, u2);
                    if (hasW) {                                             // a -> (r+1, ca-1)
                        const Cell Bn = ring_cell(chn, rn, xa - 1, hn);
                        edge<2>(a, A0, Bn, kl2, oA, pq, p1, p2);
                    } else if (own) {
                        bnd(a, A0, 2, ASX_SIDE_W, r, kl2, cA, outd);
                    }
                }
                if (vb) {
                    edge<1>(a, B0, B1, kl2, oB, q, u1, u2);             // b -> nxt b
                    if (nown) acc_in(nB, q, u1, u2);
                    edge<2>(a, B0, A1, kl2, oB, q, u1, u2);             // b -> nxt a
                    if (nown) acc_in(nA, q, u1, u2);
                } else if (va && nown) {
                    // nxt a's SE neighbour (r, cb) is beyond the east side
                    bnd(a, A1, 5, ASX_SIDE_E, r + 1, kl2, nA, outd);
                }
                // nxt b's SE neighbour (r, cb+1): the next thread's a, or beyond the raster
                if (vb && nown && t == kST - 1) {
                    if (hasE) {
                        const Cell Ec = ring_cell(chc, rc, xb + 1, hc);
                        edge<2>(a, Ec, B1, kl2, nullptr, q, u1, u2);
                        acc_in(nB, q, u1, u2);
                    }
                }
                if (!IN && vb && nown && !hasE) bnd(a, B1, 5, ASX_SIDE_E, r + 1, kl2, nB, outd);
            } else {
                // odd r: NE(c) = (r+1, c+1), NW(c) = (r+1, c)
                Acc *oA = own ? &cA : nullptr, *oB = own ? &cB : nullptr;
                if (va) {
                    edge<2>(a, A0, A1, kl2, oA, q, u1, u2);             // a -> nxt a
                    if (nown) acc_in(nA, q, u1, u2);
                    if (vb) {
                        edge<1>(a, A0, B1, kl2, oA, q, u1, u2);         // a -> nxt b
                        if (nown) acc_in(nB, q, u1, u2);
                    } else if (own) {
                        bnd(a, A0, 1, ASX_SIDE_E, r, kl2, cA, outd);
                    }
                }
                if (vb) {
                    edge<2>(a, B0, B1, kl2, oB, q, u1, u2);             // b -> nxt b
                    if (nown) acc_in(nB, q, u1, u2);
                    if (hasE) {                                             // b -> (r+1, cb+1)
                        const Cell Bn = ring_cell(chn, rn, xb + 1, hn);
                        edge<1>(a, B0, Bn, kl2, oB, pq, p1, p2);
                    } else if (own) {
                        bnd(a, B0, 1, ASX_SIDE_E, r, kl2, cB, outd);
                    }
                }
                // nxt a's SW neighbour (r, ca-1): the previous thread's b, or beyond the raster
                if (va && nown) {
                    if (!hasW) {
                        bnd(a, A1, 4, ASX_SIDE_W, r + 1, kl2, nA, outd);
                    } else if (t == 0) {
                        const Cell Wc = ring_cell(chc, rc, xa - 1, hc);
                        edge<1>(a, Wc, A1, kl2, nullptr, q, u1, u2);
                        acc_in(nA, q, u1, u2);
                    }
                }
            }
        }
        S.eDq[t] = pq; S.eD1[t] = p1; S.eD2[t] = p2;
        __syncthreads();                                           // S2
        if (own && va && hasW && t > 0) acc_in(cA, S.eEq[t - 1], S.eE1[t - 1], S.eE2[t - 1]);
        if (nown && in_r) {
            if (!odd) {
                if (vb && hasE && t < kST - 1) acc_in(nB, S.eDq[t + 1], S.eD1[t + 1], S.eD2[t + 1]);
            } else {
                if (va && hasW && t > 0) acc_in(nA, S.eDq[t - 1], S.eD1[t - 1], S.eD2[t - 1]);
            }
        }
        if (own) {
            // ---- finish the two cells of row r
            const size_t k0 = (size_t)r * a.pitch + ca;
            if (vb) {
                const CellNew oa = cell_update(cA.hi, cA.lo, cA.m1, cA.m2, A0.m, A0.v1, A0.v2, rtA0, kaA0,
                                               kbA0, kappa, qr, dtf, a.g, clq);
                const CellNew ob = cell_update(cB.hi, cB.lo, cB.m1, cB.m2, B0.m, B0.v1, B0.v2, rtB0, kaB0,
                                               kbB0, kappa, qr, dtf, a.g, clq);
                *reinterpret_cast<float2 *>(a.mhi[np] + k0) = make_float2(oa.hi, ob.hi);
                *reinterpret_cast<float2 *>(a.mlo[np] + k0) = make_float2(oa.lo, ob.lo);
                *reinterpret_cast<float2 *>(a.v1[np] + k0) = make_float2(oa.v1, ob.v1);
                *reinterpret_cast<float2 *>(a.v2[np] + k0) = make_float2(oa.v2, ob.v2);
                cwb = max(cwb, max(oa.cbits, ob.cbits));
            } else if (va) {
                const CellNew oa = cell_update(cA.hi, cA.lo, cA.m1, cA.m2, A0.m, A0.v1, A0.v2, rtA0, kaA0,
                                               kbA0, kappa, qr, dtf, a.g, clq);
                a.mhi[np][k0] = oa.hi;
                a.mlo[np][k0] = oa.lo;
                a.v1[np][k0] = oa.v1;
                a.v2[np][k0] = oa.v2;
                cwb = max(cwb, oa.cbits);
            }
        }
    }
    if (__syncthreads_or(timed_out)) {
        // a tensor copy did not arrive in time: flag the error, wait (bounded) for the
        // copies still in flight, and leave without finishing the step
        if (t == 0) {
            atomicOr(&a.ctl->err, kErrTimeout);
            for (int k = max(0, n_issued - kNC); k < n_issued; k++)
                mbar_wait_bounded(&S.bar[k % kNC], (unsigned)((k / kNC) & 1));
        }
        return;
    }
    reduce_and_finish<kST>(a, cwb, outd.value(), clq.value());
}

__global__ void __launch_bounds__(kST, 8) step_strip_kernel(const StepArgs a, const __grid_constant__ StripMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment: align the dynamic block by hand
    StripSmem &S = *reinterpret_cast<StripSmem *>(
        smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    if (!a.ctl->active) return;
    const int nstrips = (a.cols + kSW - 1) / kSW;
    const int strip = blockIdx.x % nstrips, rblk = blockIdx.x / nstrips;
    const int c0 = strip * kSW, r0 = rblk * a.tile_rows;
    const bool interior = c0 > 0 && c0 + kSW < a.cols && r0 > 0 && r0 + a.tile_rows < a.rows;
    if (interior) strip_tile<true>(a, maps, S, strip, rblk);
    else strip_tile<false>(a, maps, S, strip, rblk);
}

}  // namespace

size_t step_strip_smem() { return sizeof(StripSmem) + 128; }

int step_strip_blocks(int rows, int cols, int tile_rows)
{
    return ((cols + kSW - 1) / kSW) * ((rows + tile_rows - 1) / tile_rows);
}

cudaError_t step_strip_configure()
{
    return cudaFuncSetAttribute(step_strip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_strip_smem());
}

cudaError_t launch_step_strip(const StepArgs &a, const StripMaps &maps, cudaStream_t s)
{
    step_strip_kernel<<<a.nblocks, kST, step_strip_smem(), s>>>(a, maps);
    return cudaGetLastError();
}

}  // namespace asx
