// mlp.cu -- the learned surrogate: BF16 tensor-core GEMMs (tcgen05, accumulators in
// TMEM), the fused layer epilogues, the loss, the bias gradients and Adam, and the
// asx_mlp_* C ABI.
//
// The surrogate maps a scenario's slope, vegetation cover, porosity, plant drag and a
// 32-sample hyetograph (36 inputs, padded to 64) to a 128-sample outlet hydrograph through
// three hidden layers of 256 ReLU units: y = W4 r(W3 r(W2 r(W1 x + b1) + b2) + b3) + b4.
// Weights and activations are BF16, every product accumulates in FP32 in tensor memory,
// master weights and Adam moments are FP32.
//
// GEMM kernel: D[M x N] = A[M x K] . B[N x K]^T on one 128 x BN tile per CTA.  The four
// warps stage 128 x 64 of A and BN x 64 of B in shared memory in the tensor core's
// K-major core-matrix layout (8 rows x 16 bytes per core matrix), thread 0 issues the
// tcgen05.mma instructions (kind::f16, BF16 inputs, FP32 accumulate) and commits them to
// an mbarrier, and after the last chunk the warps read the accumulator out of TMEM with
// tcgen05.ld (warp w owns lanes 32w..32w+31 = rows) and apply the epilogue.  Operands are
// read through arbitrary strides, so the forward product, the input gradient and the
// weight gradient are all this one kernel.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "asx_internal.cuh"

namespace asx {

// 2-D tensor map over a BF16 matrix of `rows` rows of `cols` elements, `ld` elements
// apart (16-byte aligned base, ld a multiple of 8); boxes of box_x x box_y elements;
// out-of-range elements read as zero.  False if the driver refuses the map.  Defined in
// runtime.cu beside the other tensor-map builders.
bool make_tensor_map_bf16(CUtensorMap *m, const void *base, long long rows, long long cols, long long ld, int box_x,
                          int box_y);

namespace {

constexpr int kTM = 128;       // tile rows (TMEM lanes)
constexpr int kTK = 64;        // K chunk staged per round
constexpr int kGemmThreads = 256;   // two warps per TMEM lane quarter

// ----------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init1(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase (try_wait suspends the warp for a short interval
// each time); gives up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded1(unsigned long long *bar, unsigned parity)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// Shared-memory matrix descriptor of a K-major, non-swizzled operand: core matrices of
// 8 rows x 16 bytes; lbo = byte stride between core matrices along K, sbo = along M/N.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;                       // descriptor version of this tensor-core generation
    return d;                              // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr unsigned instr_desc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(kTM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(unsigned taddr, float *v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive accumulator columns of this thread's TMEM lane, one wait.
__device__ __forceinline__ void tc_ld32(unsigned taddr, float *v)
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------- the GEMM

// Staging of one GEMM operand: 0 = element by element through its strides (any layout);
// 1 = TMA tiles of an operand whose K index is contiguous; 2 = TMA tiles of an operand
// whose row (M or N) index is contiguous.
enum GemmStage : int { kStageStrided = 0, kStageKMajor = 1, kStageMNMajor = 2 };

struct GemmArgs {
    CUtensorMap ma, mb;            // tensor maps of A and B (staging 1 and 2)
    int M, N, K;
    int amode, bmode;              // GemmStage of A and B
    const __nv_bfloat16 *A;
    long long sam, sak;            // A(m, k) = A[m sam + k sak]
    const __nv_bfloat16 *B;
    long long sbn, sbk;            // B(n, k) = B[n sbn + k sbk]
    // epilogue: v = D (+ bias[n]); relu: v = max(v, 0); mask: v *= (mask[m ldm + n] > 0)
    const float *bias;
    int relu;
    const __nv_bfloat16 *mask;
    long long ldm;
    float *outf;                   // FP32 output (or nullptr)
    __nv_bfloat16 *outb;           // BF16 output (or nullptr)
    long long ldo;
    int *err;
};

// Byte offset of element (r, k) of an R x 64 K-major chunk in core-matrix layout.
__device__ __forceinline__ unsigned cm_off(int r, int k)
{
    return (unsigned)(((r >> 3) * (kTK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Bytes of one K chunk of both operands (A: 128 rows, B: BN rows, 64 BF16 columns each).
template <int BN>
constexpr int gemm_stage_bytes()
{
    return kTM * kTK * 2 + BN * kTK * 2;
}

// Two core-matrix images the tensor core reads and two TMA landing tiles.
template <int BN>
constexpr int gemm_smem_bytes()
{
    return 4 * gemm_stage_bytes<BN>() + 128;
}

__device__ __forceinline__ void mbar_expect_tx1(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// One box of a 2-D tensor map (x: the contiguous coordinate) into shared memory.
__device__ __forceinline__ void tma_tile(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// One K chunk of an operand P(r, k) (R rows from r0, 64 columns from k0; zero outside the
// nr x nk matrix) into the core-matrix image `cm`, from the TMA tile `raw` (modes 1 and
// 2) or from global memory (mode 0).
template <int R>
__device__ __forceinline__ void stage_operand(int mode, const unsigned char *raw, unsigned char *cm,
                                              const __nv_bfloat16 *P, long long s_r, long long s_k, int r0, int k0,
                                              int nr, int nk)
{
    const int tid = threadIdx.x;
    if (mode == kStageKMajor) {
        // raw: R rows of 64 elements (128 bytes); its 16-byte piece (r, q) is row r of core
        // matrix (r / 8, q).  The eight threads of a shared-memory phase take rows r mod 8 =
        // 0..7 at eight rotations of q, so that both the read and the write touch eight
        // distinct 16-byte bank groups.
        for (int i = tid; i < R * 8; i += kGemmThreads) {
            const int j = i & 7, grp = i >> 3;
            const int r = (grp % (R / 8)) * 8 + j, q = (j + grp / (R / 8)) & 7;
            const uint4 v = *reinterpret_cast<const uint4 *>(raw + r * 128 + q * 16);
            *reinterpret_cast<uint4 *>(cm + cm_off(r, q * 8)) = v;
        }
    } else if (mode == kStageMNMajor) {
        // raw: 64 rows (k) of R elements; piece (r, q) gathers elements k = 8q..8q+7 of row r
        const unsigned short *rw = reinterpret_cast<const unsigned short *>(raw);
        for (int i = tid; i < R * 8; i += kGemmThreads) {
            const int r = i % R, q = i / R;
            unsigned w[4];
#pragma unroll
            for (int j = 0; j < 4; j++)
                w[j] = (unsigned)rw[(8 * q + 2 * j) * R + r] | ((unsigned)rw[(8 * q + 2 * j + 1) * R + r] << 16);
            *reinterpret_cast<uint4 *>(cm + cm_off(r, q * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        for (int i = tid; i < R * kTK; i += kGemmThreads) {
            const int r = i / kTK, k = i % kTK;
            const int rr = r0 + r, kk = k0 + k;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (rr < nr && kk < nk) v = P[(long long)rr * s_r + (long long)kk * s_k];
            *reinterpret_cast<__nv_bfloat16 *>(cm + cm_off(r, k)) = v;
        }
    }
}

// D = A B^T for one 128 x BN tile per CTA, 64 columns of K per chunk.  Thread 0 keeps the
// TMA copies of the next two chunks in flight (landing tiles raw[c mod 2], completing on
// full[c mod 2]); the eight warps rearrange each landed chunk into the core-matrix image
// cm[c mod 2] (operands in mode 0 are read from global memory instead), and thread 0
// issues the chunk's four tcgen05 products, which commit to done[c mod 2] and so release
// the image two chunks later.  Every wait is bounded; after a failed wait the copies and
// products in flight are waited for (bounded) before TMEM is released, and *err is set.
template <int BN>
__global__ void __launch_bounds__(kGemmThreads) gemm_tc_kernel(const __grid_constant__ GemmArgs g)
{
    constexpr int kA = kTM * kTK * 2, kStage = gemm_stage_bytes<BN>();
    extern __shared__ __align__(128) unsigned char gsm[];
    unsigned char *base = gsm + ((128u - (su32(gsm) & 127u)) & 127u);
    __shared__ __align__(8) unsigned long long full[2], done[2];
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * BN;
    const unsigned tx = (g.amode != kStageStrided ? (unsigned)kA : 0u) +
                        (g.bmode != kStageStrided ? (unsigned)(BN * kTK * 2) : 0u);
    const int nchunks = (g.K + kTK - 1) / kTK;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init1(&full[s]);
            mbar_init1(&done[s]);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned idesc = instr_desc(BN);
    auto cm_of = [&](int s) { return base + s * kStage; };
    auto raw_of = [&](int s) { return base + (2 + s) * kStage; };
    auto issue = [&](int c) {      // thread 0: chunk c's tiles into raw[c mod 2]
        const int s = c & 1, k0 = c * kTK;
        mbar_expect_tx1(&full[s], tx);
        if (g.amode == kStageKMajor) tma_tile(raw_of(s), &g.ma, k0, m0, &full[s]);
        if (g.amode == kStageMNMajor) tma_tile(raw_of(s), &g.ma, m0, k0, &full[s]);
        if (g.bmode == kStageKMajor) tma_tile(raw_of(s) + kA, &g.mb, k0, n0, &full[s]);
        if (g.bmode == kStageMNMajor) tma_tile(raw_of(s) + kA, &g.mb, n0, k0, &full[s]);
    };
    int issued = 0, committed = 0, c = 0;
    if (tx != 0u && tid == 0)
        for (; issued < 2 && issued < nchunks; issued++) issue(issued);
    bool failed = false;
    for (; c < nchunks; c++) {
        const int s = c & 1;
        bool ok = true;
        // the image is free once chunk c - 2's products are done; the tiles have landed
        if (c >= 2) ok = mbar_wait_bounded1(&done[s], (unsigned)(((c - 2) >> 1) & 1));
        if (ok && tx != 0u) ok = mbar_wait_bounded1(&full[s], (unsigned)((c >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        stage_operand<kTM>(g.amode, raw_of(s), cm_of(s), g.A, g.sam, g.sak, m0, c * kTK, g.M, g.K);
        stage_operand<BN>(g.bmode, raw_of(s) + kA, cm_of(s) + kA, g.B, g.sbn, g.sbk, n0, c * kTK, g.N, g.K);
        // the tensor core and the next copies reach shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char *sA = cm_of(s), *sB = cm_of(s) + kA;
#pragma unroll
            for (int k = 0; k < kTK / 16; k++) {
                const unsigned long long da = smem_desc(su32(sA) + k * 256, 128, (kTK / 8) * 128);
                const unsigned long long db = smem_desc(su32(sB) + k * 256, 128, (kTK / 8) * 128);
                tc_mma(tmem, da, db, idesc, (c > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(&done[s]);
            committed = c + 1;
            if (tx != 0u && issued < nchunks) issue(issued++);   // chunk c + 2 into raw[s]
        }
    }
    // the last commit covers every product issued before it
    if (!failed && !mbar_wait_bounded1(&done[(nchunks - 1) & 1], (unsigned)(((nchunks - 1) >> 1) & 1))) failed = true;
    failed = __syncthreads_or(failed) != 0;
    if (failed && tid == 0) {
        for (int k = c; k < issued; k++) mbar_wait_bounded1(&full[k & 1], (unsigned)((k >> 1) & 1));
        for (int k = c >= 2 ? c - 2 : 0; k < committed; k++) mbar_wait_bounded1(&done[k & 1], (unsigned)((k >> 1) & 1));
        if (g.err) atomicOr(g.err, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: warp w reads TMEM lane quarter w mod 4 (tile rows 32 (w mod 4) ..
    // + 31) and the 32-column blocks w / 4, w / 4 + 2, ...  Each block passes through a
    // padded 32 x 33 float block of the spent staging memory, so that bias, ReLU, mask
    // and stores run along rows: lane j takes column j, and each store instruction
    // writes 32 consecutive columns of one row.  The block's mask values are loaded
    // before any of its stores.
    const int quarter = warp & 3, rbase = m0 + quarter * 32;
    float *blk = reinterpret_cast<float *>(base) + warp * (32 * 33);
    for (int nc = (warp >> 2) * 32; nc < BN && !failed; nc += 64) {
        float v[32];
        tc_ld32(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)nc, v);
#pragma unroll
        for (int j = 0; j < 32; j++) blk[lane * 33 + j] = v[j];
        __syncwarp();
        const int n = n0 + nc + lane;
        if (n < g.N) {
            const float bn = g.bias ? g.bias[n] : 0.0f;
            unsigned keep = 0xffffffffu;          // bit rr: row rbase + rr passes the mask
            if (g.mask) {
                // all 32 loads unconditional (rows past the matrix read its last row), so
                // that they are in flight together
                __nv_bfloat16 mk[32];
#pragma unroll
                for (int rr = 0; rr < 32; rr++) mk[rr] = g.mask[(long long)min(rbase + rr, g.M - 1) * g.ldm + n];
                keep = 0u;
#pragma unroll
                for (int rr = 0; rr < 32; rr++)
                    if (rbase + rr < g.M && __bfloat162float(mk[rr]) > 0.0f) keep |= 1u << rr;
            }
#pragma unroll
            for (int rr = 0; rr < 32; rr++) {
                if (rbase + rr < g.M) {
                    float x = blk[rr * 33 + lane];
                    if (g.bias) x += bn;
                    if (g.relu) x = fmaxf(x, 0.0f);
                    if (!((keep >> rr) & 1u)) x = 0.0f;
                    const long long o = (long long)(rbase + rr) * g.ldo + n;
                    if (g.outf) g.outf[o] = x;
                    if (g.outb) g.outb[o] = __float2bfloat16(x);
                }
            }
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// ----------------------------------------------------------------- small kernels

// db[n] = sum_m dZ[m][n] (FP32 from the BF16 gradient).  A block of 32 x 32 threads takes
// 32 columns: thread (x, y) sums rows y, y + 32, y + 64, ... of column x in that order and
// the threads of row 0 add the 32 partial sums in order of y, a fixed order, so the
// result is the same on every run.  Launched with kBiasGradThreads threads per block.
constexpr int kBiasGradThreads = 1024;
__global__ void __launch_bounds__(kBiasGradThreads) bias_grad_kernel(const __nv_bfloat16 *dz, int M, int N, float *db)
{
    __shared__ float part[32][33];
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + x;
    float s = 0.0f;
    if (n < N)
        for (int m = y; m < M; m += 32) s += __bfloat162float(dz[(long long)m * N + n]);
    part[y][x] = s;
    __syncthreads();
    if (y == 0 && n < N) {
        float t = 0.0f;
        for (int k = 0; k < 32; k++) t += part[k][x];
        db[n] = t;
    }
}

// Mean-squared error over a batch and its gradient dY = 2 (Y - T) / (M N) as BF16.
__global__ void mse_grad_kernel(const float *y, const float *t, int n_elem, float scale, __nv_bfloat16 *dy,
                                float *loss_acc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < n_elem) {
        const float d = y[i] - t[i];
        l = d * d;
        dy[i] = __float2bfloat16(2.0f * d * scale);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss_acc, l * scale);
}

// Adam on FP32 master weights over up to kAdamSegs segments in one launch (element i of
// the launch belongs to the segment s with start[s] <= i < start[s + 1]), refreshing the
// BF16 copy where a segment has one; decay wd per segment.
constexpr int kAdamSegs = 8;
struct AdamArgs {
    float *w[kAdamSegs];
    const float *grad[kAdamSegs];
    float *mo[kAdamSegs], *ve[kAdamSegs];
    __nv_bfloat16 *wb[kAdamSegs];
    float wd[kAdamSegs];
    int start[kAdamSegs + 1];
    int nseg;
    float lr, b1, b2, eps, c1, c2;
};

__global__ void adam_kernel(const AdamArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.start[a.nseg]) return;
    int sg = 0;
    while (t >= a.start[sg + 1]) sg++;
    const int i = t - a.start[sg];
    float *w = a.w[sg], *mo = a.mo[sg], *ve = a.ve[sg];
    const float *grad = a.grad[sg];
    __nv_bfloat16 *wb = a.wb[sg];
    const float wd = a.wd[sg], lr = a.lr, b1 = a.b1, b2 = a.b2, eps = a.eps, c1 = a.c1, c2 = a.c2;
    const float gi = grad[i] + wd * w[i];
    const float m = b1 * mo[i] + (1.0f - b1) * gi;
    const float v = b2 * ve[i] + (1.0f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    const float x = w[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    w[i] = x;
    if (wb) wb[i] = __float2bfloat16(x);
}

__global__ void f32_to_bf16_kernel(const float *x, __nv_bfloat16 *y, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

// x (M x din FP32, row-major) -> (M x ldx BF16) with zero padding of the extra columns.
__global__ void pad_input_kernel(const float *x, int M, int din, int ldx, __nv_bfloat16 *y)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * ldx) return;
    const int m = (int)(i / ldx), k = (int)(i % ldx);
    y[i] = __float2bfloat16(k < din ? x[(long long)m * din + k] : 0.0f);
}


// The surrogate's error check (one warp per checked query): e_k = ||y_q - ref_k|| /
// ||ref_k|| over the hydrograph's samples, q = idx[k]; where e_k > tol (or is not a
// number) the solver's hydrograph replaces the surrogate's in y.  An index outside
// [0, batch) is skipped and reported as NaN.
__global__ void hydro_check_kernel(int batch, int n_check, int len, const int *__restrict__ idx, float *y,
                                   const float *__restrict__ ref, float tol, float *rel_err, int *n_replaced)
{
    const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n_check) return;
    const int q = idx[k];
    if (q < 0 || q >= batch) {
        if (lane == 0) rel_err[k] = __int_as_float(0x7fc00000);
        return;
    }
    float *yq = y + (size_t)q * len;
    const float *rk = ref + (size_t)k * len;
    double dd = 0.0, rr = 0.0;
    for (int j = lane; j < len; j += 32) {
        const double d = (double)yq[j] - (double)rk[j];
        dd += d * d;
        rr += (double)rk[j] * (double)rk[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
    }
    const float e = rr > 0.0 ? (float)sqrt(dd / rr) : (dd > 0.0 ? __int_as_float(0x7f800000) : 0.0f);
    const bool replace = !(e <= tol);
    if (replace)
        for (int j = lane; j < len; j += 32) yq[j] = rk[j];
    if (lane == 0) {
        rel_err[k] = e;
        if (replace) atomicAdd(n_replaced, 1);
    }
}
}  // namespace

// Staging of an operand P(r, k) = P[r s_r + k s_k] of R rows and K columns: TMA tiles of
// box_r rows x 64 columns where its layout allows them (16-byte aligned base, one unit
// stride, the other a multiple of 8 elements and at least the contiguous extent), with
// the tensor map in *map; element by element otherwise.
int stage_mode(CUtensorMap *map, const __nv_bfloat16 *P, long long s_r, long long s_k, int R, int K, int box_r)
{
    if ((reinterpret_cast<uintptr_t>(P) & 15u) != 0) return kStageStrided;
    if (s_k == 1 && s_r % 8 == 0 && s_r >= K && make_tensor_map_bf16(map, P, R, K, s_r, kTK, box_r))
        return kStageKMajor;
    if (s_r == 1 && s_k % 8 == 0 && s_k >= R && make_tensor_map_bf16(map, P, K, R, s_k, box_r, kTK))
        return kStageMNMajor;
    return kStageStrided;
}

template <int BN>
cudaError_t launch_gemm_bn(const GemmArgs &g0, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             gemm_smem_bytes<BN>());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    GemmArgs g = g0;
    g.amode = stage_mode(&g.ma, g.A, g.sam, g.sak, g.M, g.K, kTM);
    g.bmode = stage_mode(&g.mb, g.B, g.sbn, g.sbk, g.N, g.K, BN);
    dim3 grid((g.M + kTM - 1) / kTM, (g.N + BN - 1) / BN);
    gemm_tc_kernel<BN><<<grid, kGemmThreads, gemm_smem_bytes<BN>(), s>>>(g);
    return cudaGetLastError();
}

// Tile width: 256 (or 128 for N <= 128) where the grid of such tiles already gives about
// one CTA per SM, else 64, for up to four times the CTAs: a small GEMM is bound by the
// latency of each CTA's staging and epilogue, not by the tensor pipe.
cudaError_t launch_gemm_tc(const GemmArgs &g, cudaStream_t s)
{
    const long long mt = (g.M + kTM - 1) / kTM;
    if (g.N > 128 && mt * ((g.N + 255) / 256) >= 128) return launch_gemm_bn<256>(g, s);
    if (g.N > 64 && mt * ((g.N + 127) / 128) >= 128) return launch_gemm_bn<128>(g, s);
    return launch_gemm_bn<64>(g, s);
}

}  // namespace asx

using namespace asx;

// ------------------------------------------------------------------ C ABI

extern "C" asx_status asx_gemm_bf16(int M, int N, int K, const void *A, long long sam, long long sak, const void *B,
                                    long long sbn, long long sbk, float *D, long long ldd, void *cuda_stream)
{
    if (M < 1 || N < 1 || K < 1 || !A || !B || !D || ldd < N) return ASX_EINVAL;
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = static_cast<const __nv_bfloat16 *>(A);
    g.sam = sam;
    g.sak = sak;
    g.B = static_cast<const __nv_bfloat16 *>(B);
    g.sbn = sbn;
    g.sbk = sbk;
    g.outf = D;
    g.ldo = ldd;
    return launch_gemm_tc(g, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? ASX_OK : ASX_ECUDA;
}

// ------------------------------------------------------------------ the MLP

namespace asx {
namespace {

constexpr int kIn = ASX_MLP_IN, kInPad = 64, kHid = ASX_MLP_HIDDEN, kOut = ASX_MLP_OUT;

// Offsets (in floats) of the padded parameter layout: W1 is kept 256 x 64 with zero
// columns 36..63 (their gradient is zero, so Adam keeps them zero).
constexpr long long oW1 = 0, oB1 = oW1 + (long long)kHid * kInPad, oW2 = oB1 + kHid, oB2 = oW2 + (long long)kHid * kHid,
                    oW3 = oB2 + kHid, oB3 = oW3 + (long long)kHid * kHid, oW4 = oB3 + kHid,
                    oB4 = oW4 + (long long)kOut * kHid, kPadded = oB4 + kOut;

}  // namespace
}  // namespace asx

namespace asx {
namespace {

// ----------------------------------------------------------------- the fused forward pass
//
// One CTA (sixteen warps) carries two tiles of 128 queries (a pair) through all four
// layers.  The input tiles (BF16, K padded to 64) and the activations (128 x 256 BF16 per
// tile) stay in shared memory in the tensor core's core-matrix layout; each tile's
// products accumulate in its own 256-column TMEM accumulator (512 columns for the pair),
// and each layer's epilogue (bias, ReLU, BF16) writes the next layer's operand straight
// back to shared memory.  The weights stream through a ring of two 32 KB slots, one K = 64
// chunk of a layer's weight matrix per slot, copied from an image kept in exactly the
// shared-memory layout (cp.async.bulk on an mbarrier); each chunk feeds both tiles, so a
// pair reads the 352 KB of weights once (thirteen chunks: W1, W2 x 4, W3 x 4, W4 x 4).
// One thread issues the copies and the products: chunk g's products are queued before it
// waits for chunk g-1's to finish and refills that slot with chunk g+1, so a copy runs
// under the products of the chunk before it; at a layer's end the next layer's first
// chunks load during the epilogue.  CTAs are persistent over the pairs.  Shared memory:
// 2 x 16 KB inputs + 2 x 64 KB activations + 64 KB ring.

// 18 warps: warp 0 issues the products, warp 1 the weight copies, warps 2..17 stage the
// inputs and run the epilogues; warp w reads TMEM lanes 32 (w % 4) .. +31 (the hardware's
// lane quarter of a warp) and a quarter of the columns, (w - 2) / 4.
constexpr int kEpiWarps = 16;
constexpr int kFusedThreads = 32 * (2 + kEpiWarps);
constexpr int kColGroups = 4;
constexpr unsigned kWtBytes1 = (unsigned)kHid * kInPad * 2;   // W1: 32 KB
constexpr unsigned kWtBytesH = (unsigned)kHid * kHid * 2;     // W2, W3: 128 KB each
constexpr unsigned kWtBytes4 = (unsigned)kOut * kHid * 2;     // W4: 64 KB
constexpr unsigned kWtOff1 = 0, kWtOff2 = kWtBytes1, kWtOff3 = kWtOff2 + kWtBytesH, kWtOff4 = kWtOff3 + kWtBytesH;
constexpr unsigned kWtTotal = kWtOff4 + kWtBytes4;
constexpr int kSmX = kTM * kInPad * 2;                        // 16 KB per tile
constexpr int kSmAct = kTM * kHid * 2;                        // 64 KB per tile
constexpr int kCK = 64;                                       // K columns of a weight chunk
constexpr int kNSlot = 2;                                     // ring slots
constexpr unsigned kSlot = (unsigned)kHid * kCK * 2;          // 32 KB: one chunk of 256 rows
constexpr int kChunksPerPair = (kInPad + 3 * kHid) / kCK;     // 13: W1, then W2, W3, W4 by K chunks
constexpr int kFusedSmem = 2 * kSmX + 2 * kSmAct + kNSlot * (int)kSlot + 128;
static_assert(kFusedSmem <= 232448, "shared memory per CTA");

// Chunk jj of a pair's weight stream: its layer, the chunk's index in the layer, byte
// offset in the image (the image is laid out in stream order) and size.
__device__ __forceinline__ void weight_chunk(int jj, int &layer, int &c, unsigned &off, unsigned &bytes)
{
    constexpr int n1 = kInPad / kCK, nh = kHid / kCK;
    if (jj < n1) {
        layer = 0;
        c = jj;
        off = kWtOff1 + (unsigned)c * kSlot;
        bytes = kSlot;
    } else if (jj < n1 + 2 * nh) {
        layer = 1 + (jj - n1) / nh;
        c = (jj - n1) % nh;
        off = kWtOff2 + (unsigned)(jj - n1) * kSlot;
        bytes = kSlot;
    } else {
        layer = 3;
        c = jj - n1 - 2 * nh;
        off = kWtOff4 + (unsigned)c * (unsigned)(kOut * kCK * 2);
        bytes = (unsigned)(kOut * kCK * 2);
    }
}

// Byte offset of element (r, k) of an R-row K-major operand stored as K/64 chunks of
// R x 64 in core-matrix layout (chunk c at c * R * 128 bytes).
__device__ __forceinline__ unsigned cm_off_k(int R, int r, int k)
{
    return (unsigned)((k >> 6) * R * 128) + cm_off(r, k & 63);
}

// The same for the weight image's chunks of kCK columns: chunk c at c * R * kCK * 2 bytes,
// core matrices of 8 rows x 16 bytes, kCK / 8 of them along K per 8-row group.
__device__ __forceinline__ unsigned cm_off_w(int R, int r, int k)
{
    const int c = k / kCK, kk = k % kCK;
    return (unsigned)(c * R * kCK * 2 + ((r >> 3) * (kCK / 8) + (kk >> 3)) * 128 + (r & 7) * 16 + (kk & 7) * 2);
}

// The BF16 weights (row-major N x K, W1 | W2 | W3 | W4) into the image the fused kernel
// copies to shared memory; 8 consecutive k of one row (16 bytes) per thread.
__global__ void tile_weights_kernel(const __nv_bfloat16 *wb, unsigned char *wt)
{
    long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long src = 0, dst = 0;
#pragma unroll
    for (int l = 0; l < 4; l++) {
        const int N = l == 3 ? kOut : kHid, K = l == 0 ? kInPad : kHid;
        const long long units = (long long)N * K / 8;
        if (u < units) {
            const int r = (int)(u / (K / 8)), k = (int)(u % (K / 8)) * 8;
            const uint4 v = *reinterpret_cast<const uint4 *>(wb + src + (long long)r * K + k);
            *reinterpret_cast<uint4 *>(wt + dst + cm_off_w(N, r, k)) = v;
            return;
        }
        u -= units;
        src += (long long)N * K;
        dst += (long long)N * K * 2;
    }
}

struct FusedArgs {
    const float *x;                // batch x 36 FP32, rows 16-byte aligned
    float *y;                      // batch x 128 FP32, 16-byte aligned
    const unsigned char *wt;       // weight image, kWtTotal bytes
    const float *b1, *b2, *b3, *b4;
    int batch;
    int *err;
};

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, at most 32 KB, both addresses
// 16-byte aligned) completing on `bar`; one thread.
__device__ __forceinline__ void load_chunk(unsigned char *dst, const unsigned char *src, unsigned bytes,
                                           unsigned long long *bar)
{
    mbar_expect(bar, bytes);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

// BF16 pair of ReLU(a + b) (element 0 in the low half): a packed float32 add (each
// component rounded as the scalar add), round to nearest even, then the maximum with zero
// on the BF16 pair (rounding is monotone and keeps zero, so this is ReLU before rounding).
__device__ __forceinline__ unsigned bias_relu_bf16x2(float a0, float a1, float b0, float b1)
{
    unsigned r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t.reg .f32 s0, s1;\n\t.reg .b32 h, z;\n\t"
        "mov.b64 ra, {%1, %2};\n\tmov.b64 rb, {%3, %4};\n\tadd.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {s0, s1}, rd;\n\tcvt.rn.bf16x2.f32 h, s1, s0;\n\tmov.b32 z, 0;\n\t"
        "max.bf16x2 %0, h, z;\n\t}"
        : "=r"(r)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
    return r;
}

// Hidden-layer epilogue of accumulator row r (this thread's TMEM lane) of the nt tiles,
// columns [c0, c1) (a multiple of 32): + bias, ReLU, BF16 (round to nearest even), into
// each tile's activation image.  The biases are loaded once for the tiles.
__device__ __forceinline__ void epi_hidden(unsigned trow, int nt, const float *__restrict__ bias,
                                           unsigned char *const *act, int r, int c0, int c1)
{
    for (int nc = c0; nc < c1; nc += 32) {
        float bv[32];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 b = __ldg(reinterpret_cast<const float4 *>(bias + nc) + q);
            bv[4 * q] = b.x;
            bv[4 * q + 1] = b.y;
            bv[4 * q + 2] = b.z;
            bv[4 * q + 3] = b.w;
        }
        for (int t = 0; t < nt; t++) {
            float v[32];
            tc_ld32(trow + (unsigned)(t * kHid + nc), v);
            unsigned w[16];
#pragma unroll
            for (int j = 0; j < 16; j++) w[j] = bias_relu_bf16x2(v[2 * j], v[2 * j + 1], bv[2 * j], bv[2 * j + 1]);
#pragma unroll
            for (int g8 = 0; g8 < 4; g8++)
                *reinterpret_cast<uint4 *>(act[t] + cm_off_k(kTM, r, nc + 8 * g8)) =
                    make_uint4(w[4 * g8], w[4 * g8 + 1], w[4 * g8 + 2], w[4 * g8 + 3]);
        }
    }
}

// Output epilogue of one tile: + bias, FP32, rows m0 .. m0 + 127 of y.  Each warp owns 32
// rows (its TMEM lanes) x 32 columns: it passes them through a 32 x 32 block of shared
// memory (4 KB; 16-byte chunk q of row r stored at chunk q ^ (r & 7), so that eight lanes'
// 16-byte accesses hit 32 distinct banks), and each store instruction writes four rows of
// 32 consecutive floats.
__device__ __forceinline__ void epi_output(unsigned trow, const float *__restrict__ bias, float *stage, float *y,
                                           int m0, int batch, int quarter, int cgroup)
{
    const int lane = threadIdx.x & 31, c0 = cgroup * 32;
    float v[32];
    tc_ld32(trow + (unsigned)c0, v);
    float4 *srow = reinterpret_cast<float4 *>(stage + lane * 32);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const float4 b = __ldg(reinterpret_cast<const float4 *>(bias + c0) + q);
        srow[q ^ (lane & 7)] = make_float4(v[4 * q] + b.x, v[4 * q + 1] + b.y, v[4 * q + 2] + b.z, v[4 * q + 3] + b.w);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int rr = 4 * i + (lane >> 3), q = lane & 7;
        const int m = m0 + quarter * 32 + rr;
        const float4 val = reinterpret_cast<const float4 *>(stage + rr * 32)[q ^ (rr & 7)];
        if (m < batch) reinterpret_cast<float4 *>(y + (size_t)m * kOut + c0)[q] = val;
    }
    __syncwarp();
}

__device__ __forceinline__ void mbar_arrive1(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait that also gives up when another role has failed (*fail set).
__device__ __forceinline__ bool wait_or_fail(unsigned long long *bar, unsigned parity, volatile int *fail)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*fail || global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// The weight stream of one CTA (issued by one thread): chunk j of the stream is chunk
// j mod 13 of a pair's sequence, in ring slot j mod 2.
struct WeightStream {
    const unsigned char *wt;
    unsigned char *ring;
    unsigned long long *full, *empty;   // per slot: copy landed / products done with it
    int total;                          // chunks this CTA consumes
    int issued = 0, freed = 0;          // chunks copied / known to be free again
    bool ok = true;

    // Copy every chunk whose slot is free, up to kNSlot ahead of the products.
    __device__ __forceinline__ void refill()
    {
        while (issued < total && issued - freed < kNSlot) {
            int layer, c;
            unsigned off, bytes;
            weight_chunk(issued % kChunksPerPair, layer, c, off, bytes);
            load_chunk(ring + (issued % kNSlot) * kSlot, wt + off, bytes, &full[issued % kNSlot]);
            issued++;
        }
    }
    // Wait until the products of chunks up to j are done with their slots.
    __device__ __forceinline__ void free_through(int j)
    {
        while (ok && freed <= j) {
            ok = mbar_wait_bounded1(&empty[freed % kNSlot], (unsigned)((freed / kNSlot) & 1));
            if (ok) freed++;
        }
    }
};

__global__ void __launch_bounds__(kFusedThreads, 1) mlp_fused_fwd_kernel(const FusedArgs f)
{
    extern __shared__ __align__(128) unsigned char fsm[];
    unsigned char *base = fsm + ((128u - (su32(fsm) & 127u)) & 127u);
    unsigned char *sX[2] = {base, base + kSmX};
    unsigned char *sAct[2] = {base + 2 * kSmX, base + 2 * kSmX + kSmAct};
    unsigned char *sW = base + 2 * kSmX + 2 * kSmAct;
    // full / empty: the weight ring; acc[t]: tile t's products of a layer are done;
    // epi[t]: tile t's hidden epilogue is done (16 arrivals); xrdy: a pair's inputs are
    // staged (16 arrivals)
    __shared__ __align__(8) unsigned long long bar_full[kNSlot], bar_empty[kNSlot], bar_acc[2], bar_epi[2], bar_x;
    __shared__ unsigned tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (f.batch + kTM - 1) / kTM, npairs = (ntiles + 1) / 2;
    const int my_pairs = (int)blockIdx.x < npairs ? (npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(2 * kHid)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < kNSlot; k++) {
            mbar_init1(&bar_full[k]);
            mbar_init1(&bar_empty[k]);
        }
        for (int t = 0; t < 2; t++) {
            mbar_init1(&bar_acc[t]);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar_epi[t])), "r"(kEpiWarps) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar_x)), "r"(kEpiWarps) : "memory");
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    volatile int *fail = &s_fail;
    if (warp == 0) {
        // ---- products (one thread)
        if (lane == 0) {
            int g = 0;                         // first chunk of the running layer
            unsigned px = 0, pe[2] = {0, 0};   // phases of bar_x and bar_epi
            bool ok = true;
            for (int pi = 0; pi < my_pairs && ok; pi++) {
                const int nt = min(2, ntiles - 2 * ((int)blockIdx.x + pi * (int)gridDim.x));
                ok = wait_or_fail(&bar_x, px, fail);            // this pair's inputs are staged
                px ^= 1u;
                for (int l = 0; l < 4 && ok; l++) {
                    const int nch = (l == 0 ? kInPad : kHid) / kCK;
                    const unsigned idesc = instr_desc(l == 3 ? kOut : kHid);
                    for (int c = 0; c < nch && ok; c++) {
                        const int gg = g + c;
                        ok = wait_or_fail(&bar_full[gg % kNSlot], (unsigned)((gg / kNSlot) & 1), fail);
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const unsigned bw = su32(sW + (gg % kNSlot) * kSlot);
                        for (int t = 0; t < nt && ok; t++) {
                            if (c == 0 && (l > 0 || pi > 0)) {
                                // tile t's operand and accumulator are free once its previous
                                // epilogue (the last pair's output, for the first layer) is
                                // done; the other tile's epilogue may still run
                                ok = wait_or_fail(&bar_epi[t], pe[t], fail);
                                pe[t] ^= 1u;
                                if (!ok) break;
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            }
                            const unsigned ab = su32(l == 0 ? sX[t] : sAct[t]);
                            for (int s = 0; s < kCK / 16; s++) {
                                // A: K columns c kCK + 16 s .. +15 of the tile's K/64-chunked operand
                                const int k = c * kCK + 16 * s;
                                const unsigned long long da = smem_desc(
                                    ab + (unsigned)((k >> 6) * kTM * 128 + ((k & 63) >> 3) * 128), 128, 1024);
                                const unsigned long long db = smem_desc(bw + (unsigned)(s * 256), 128, kCK / 8 * 128);
                                tc_mma(tmem + (unsigned)(t * kHid), da, db, idesc, (c > 0 || s > 0) ? 1u : 0u);
                            }
                            if (c == nch - 1) tc_commit(&bar_acc[t]);   // tile t's layer is done
                        }
                        if (ok) tc_commit(&bar_empty[gg % kNSlot]);
                    }
                    g += nch;
                }
            }
            if (!ok) {
                // let every product issued land before the tensor memory is released
                *fail = 1;
                tc_commit(&bar_empty[0]);
                mbar_wait_bounded1(&bar_empty[0], 0u);
                mbar_wait_bounded1(&bar_empty[0], 1u);
            }
        }
    } else if (warp == 1) {
        // ---- weight copies (one thread): free each chunk's slot when its products are
        // done and refill the ring
        if (lane == 0) {
            WeightStream ws;
            ws.wt = f.wt;
            ws.ring = sW;
            ws.full = bar_full;
            ws.empty = bar_empty;
            ws.total = my_pairs * kChunksPerPair;
            ws.refill();
            for (int j = 0; j < ws.total && ws.ok && !*fail; j++) {
                ws.free_through(j);
                ws.refill();
            }
            if (!ws.ok || *fail) {
                *fail = 1;
                for (int j = ws.freed; j < ws.issued; j++)
                    mbar_wait_bounded1(&bar_full[j % kNSlot], (unsigned)((j / kNSlot) & 1));
            }
        }
    } else {
        // ---- input staging and epilogues (warps 2..17)
        const int quarter = warp & 3, cgroup = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;                  // this thread's accumulator row
        const unsigned trow = tmem + ((unsigned)(quarter * 32) << 16);
        const float *bias[3] = {f.b1, f.b2, f.b3};
        unsigned pa[2] = {0, 0};                              // phases of bar_acc
        bool ok = true;
        // input tiles of pair pi to BF16, K padded to 64: one (row, 8-column group) per
        // thread and pass; then this warp's share is announced on bar_x
        auto stage_inputs = [&](int pi) {
            const int m0 = ((int)blockIdx.x + pi * (int)gridDim.x) * 2 * kTM;
            for (int u = tid - 64; u < 2 * kTM * (kInPad / 8); u += 32 * kEpiWarps) {
                const int r = u % (2 * kTM), kg = u / (2 * kTM), m = m0 + r;
                float xv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                if (m < f.batch && kg * 8 < kIn) {
                    const float4 *xr = reinterpret_cast<const float4 *>(f.x + (size_t)m * kIn + kg * 8);
                    const float4 a4 = xr[0];
                    xv[0] = a4.x;
                    xv[1] = a4.y;
                    xv[2] = a4.z;
                    xv[3] = a4.w;
                    if (kg * 8 + 4 < kIn) {
                        const float4 b4v = xr[1];
                        xv[4] = b4v.x;
                        xv[5] = b4v.y;
                        xv[6] = b4v.z;
                        xv[7] = b4v.w;
                    }
                }
                unsigned w[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(xv[2 * j], xv[2 * j + 1]);
                    w[j] = *reinterpret_cast<const unsigned *>(&h);
                }
                *reinterpret_cast<uint4 *>(sX[r >> 7] + cm_off(r & (kTM - 1), kg * 8)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive1(&bar_x);
        };
        if (my_pairs > 0) stage_inputs(0);
        for (int pi = 0; pi < my_pairs && ok; pi++) {
            const int pair = (int)blockIdx.x + pi * (int)gridDim.x;
            const int m0 = pair * 2 * kTM;
            const int nt = min(2, ntiles - 2 * pair);
            for (int l = 0; l < 4 && ok; l++) {
                for (int t = 0; t < nt && ok; t++) {
                    ok = wait_or_fail(&bar_acc[t], pa[t], fail);
                    pa[t] ^= 1u;
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (l < 3) {
                        unsigned char *act[1] = {sAct[t]};
                        epi_hidden(trow + (unsigned)(t * kHid), 1, bias[l], act, row, cgroup * (kHid / kColGroups),
                                   (cgroup + 1) * (kHid / kColGroups));
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    } else {
                        // the tile's activations are spent: their buffer holds the warps'
                        // 32 x 32 output blocks
                        epi_output(trow + (unsigned)(t * kHid), f.b4,
                                   reinterpret_cast<float *>(sAct[t]) + (warp - 2) * 32 * 32, f.y, m0 + t * kTM, f.batch,
                                   quarter, cgroup);
                    }
                    // tile t's accumulator is read (and, below the output layer, its next
                    // operand written)
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive1(&bar_epi[t]);
                }
                // the first layer's products are done with the inputs: stage the next pair's
                if (l == 0 && ok && pi + 1 < my_pairs) stage_inputs(pi + 1);
            }
        }
        if (!ok) *fail = 1;
    }
    __syncthreads();
    if (s_fail && tid == 0 && f.err) atomicOr(f.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kHid) : "memory");
    }
}

}  // namespace
}  // namespace asx

struct asx_mlp {
    int device = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 master, grad, Adam moments
    __nv_bfloat16 *wb = nullptr;                                    // BF16 copies of W1..W4 (padded layout)
    unsigned char *wt = nullptr;                                    // the same in the fused kernel's image
    bool wt_dirty = true;                                           // wt lags behind wb
    int n_sm = 0;
    __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dy = nullptr, *dz = nullptr,
                  *dz2 = nullptr;
    float *y = nullptr, *xin = nullptr, *tin = nullptr, *loss = nullptr;
    int *err = nullptr;
    long long adam_t = 0;
    // The training step's kernels after its input copies, as a CUDA graph per batch size:
    // captured (on the private stream cap) at the second step with that batch size, the
    // first having run them eagerly; exec null where capture was not possible.  Each
    // launch first sets the Adam node's scalars.
    struct TrainGraph {
        int batch;
        cudaGraph_t graph;             // kept: the Adam node's handle belongs to it
        cudaGraphExec_t exec;
        cudaGraphNode_t adam;
        cudaKernelNodeParams kp;
    };
    std::vector<TrainGraph> graphs;
    std::vector<int> seen;
    cudaStream_t cap = nullptr;
    std::string error;
};

namespace {

using namespace asx;

asx_status mfail(asx_mlp *p, asx_status st, const std::string &s)
{
    if (p) p->error = s;
    return st;
}

#define MLP_CUDA(p, call)                                                                        \
    do {                                                                                         \
        cudaError_t x_ = (call);                                                                 \
        if (x_ != cudaSuccess)                                                                   \
            return mfail((p), ASX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(x_));    \
    } while (0)

GemmArgs gemm(int M, int N, int K, const __nv_bfloat16 *A, long long sam, long long sak, const __nv_bfloat16 *B,
              long long sbn, long long sbk, int *err)
{
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.sam = sam;
    g.sak = sak;
    g.B = B;
    g.sbn = sbn;
    g.sbk = sbk;
    g.err = err;
    return g;
}

__nv_bfloat16 *wb_of(asx_mlp *p, int layer)
{
    static const long long off[4] = {oW1, oW2 - kHid, oW3 - 2 * kHid, oW4 - 3 * kHid};
    return p->wb + off[layer];
}

// Forward pass of `batch` rows already in p->x0 (BF16, padded); fills a1..a3 and y.
cudaError_t forward(asx_mlp *p, int B)
{
    GemmArgs g = gemm(B, kHid, kInPad, p->x0, kInPad, 1, wb_of(p, 0), kInPad, 1, p->err);
    g.bias = p->w + oB1;
    g.relu = 1;
    g.outb = p->a1;
    g.ldo = kHid;
    cudaError_t e = launch_gemm_tc(g, p->stream);
    if (e != cudaSuccess) return e;
    const __nv_bfloat16 *in[2] = {p->a1, p->a2};
    __nv_bfloat16 *out[2] = {p->a2, p->a3};
    const long long ob[2] = {oB2, oB3};
    for (int l = 0; l < 2; l++) {
        g = gemm(B, kHid, kHid, in[l], kHid, 1, wb_of(p, l + 1), kHid, 1, p->err);
        g.bias = p->w + ob[l];
        g.relu = 1;
        g.outb = out[l];
        g.ldo = kHid;
        e = launch_gemm_tc(g, p->stream);
        if (e != cudaSuccess) return e;
    }
    g = gemm(B, kOut, kHid, p->a3, kHid, 1, wb_of(p, 3), kHid, 1, p->err);
    g.bias = p->w + oB4;
    g.outf = p->y;
    g.ldo = kOut;
    return launch_gemm_tc(g, p->stream);
}

// Gradients of the mean-squared error of the last forward pass against targets p->tin
// into p->g (padded layout); the loss into p->loss[0].
cudaError_t backward(asx_mlp *p, int B)
{
    cudaError_t e = cudaMemsetAsync(p->loss, 0, sizeof(float), p->stream);
    if (e != cudaSuccess) return e;
    const int ne = B * kOut;
    mse_grad_kernel<<<(ne + 255) / 256, 256, 0, p->stream>>>(p->y, p->tin, ne, 1.0f / (float)ne, p->dy, p->loss);
    // layer 4
    GemmArgs g = gemm(kOut, kHid, B, p->dy, 1, kOut, p->a3, 1, kHid, p->err);   // dW4 = dY^T A3
    g.outf = p->g + oW4;
    g.ldo = kHid;
    if ((e = launch_gemm_tc(g, p->stream)) != cudaSuccess) return e;
    bias_grad_kernel<<<(kOut + 31) / 32, kBiasGradThreads, 0, p->stream>>>(p->dy, B, kOut, p->g + oB4);
    g = gemm(B, kHid, kOut, p->dy, kOut, 1, wb_of(p, 3), 1, kHid, p->err);      // dZ3 = (dY W4) r'(z3)
    g.mask = p->a3;
    g.ldm = kHid;
    g.outb = p->dz;
    g.ldo = kHid;
    if ((e = launch_gemm_tc(g, p->stream)) != cudaSuccess) return e;
    // layers 3 and 2
    const __nv_bfloat16 *act_in[2] = {p->a2, p->a1};
    const long long ow[2] = {oW3, oW2}, ob[2] = {oB3, oB2};
    __nv_bfloat16 *cur = p->dz, *nxt = p->dz2;
    for (int l = 0; l < 2; l++) {
        g = gemm(kHid, kHid, B, cur, 1, kHid, act_in[l], 1, kHid, p->err);       // dW = dZ^T A_in
        g.outf = p->g + ow[l];
        g.ldo = kHid;
        if ((e = launch_gemm_tc(g, p->stream)) != cudaSuccess) return e;
        bias_grad_kernel<<<(kHid + 31) / 32, kBiasGradThreads, 0, p->stream>>>(cur, B, kHid, p->g + ob[l]);
        g = gemm(B, kHid, kHid, cur, kHid, 1, wb_of(p, 2 - l), 1, kHid, p->err);  // dZ_in = (dZ W) r'
        g.mask = act_in[l];
        g.ldm = kHid;
        g.outb = nxt;
        g.ldo = kHid;
        if ((e = launch_gemm_tc(g, p->stream)) != cudaSuccess) return e;
        __nv_bfloat16 *t = cur;
        cur = nxt;
        nxt = t;
    }
    // layer 1
    g = gemm(kHid, kInPad, B, cur, 1, kHid, p->x0, 1, kInPad, p->err);           // dW1 = dZ1^T X
    g.outf = p->g + oW1;
    g.ldo = kInPad;
    if ((e = launch_gemm_tc(g, p->stream)) != cudaSuccess) return e;
    bias_grad_kernel<<<(kHid + 31) / 32, kBiasGradThreads, 0, p->stream>>>(cur, B, kHid, p->g + oB1);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(asx_mlp *p)
{
    const long long segs[4][2] = {{oW1, (long long)kHid * kInPad}, {oW2, (long long)kHid * kHid},
                                  {oW3, (long long)kHid * kHid}, {oW4, (long long)kOut * kHid}};
    for (int l = 0; l < 4; l++) {
        const long long n = segs[l][1];
        f32_to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(p->w + segs[l][0], wb_of(p, l), n);
    }
    return cudaGetLastError();
}

// Packed (public) <-> padded (internal) parameter layouts on the host.
void pack_to_padded(const float *src, std::vector<float> &dst)
{
    dst.assign((size_t)kPadded, 0.0f);
    const float *s = src;
    for (int o = 0; o < kHid; o++)
        for (int i = 0; i < kIn; i++) dst[oW1 + (long long)o * kInPad + i] = *s++;
    std::memcpy(&dst[oB1], s, sizeof(float) * (size_t)(kPadded - oB1));
}

void padded_to_pack(const std::vector<float> &src, float *dst)
{
    float *d = dst;
    for (int o = 0; o < kHid; o++)
        for (int i = 0; i < kIn; i++) *d++ = src[oW1 + (long long)o * kInPad + i];
    std::memcpy(d, &src[oB1], sizeof(float) * (size_t)(kPadded - oB1));
}

// Forward pass of B queries x (device, 16-byte aligned) into y (device, 16-byte aligned)
// by the fused kernel; refreshes the weight image first when the weights changed.
cudaError_t fused_forward(asx_mlp *p, int B, const float *x, float *y)
{
    if (p->wt_dirty) {
        const long long units = ((long long)kHid * kInPad + 2LL * kHid * kHid + (long long)kOut * kHid) / 8;
        tile_weights_kernel<<<(unsigned)((units + 255) / 256), 256, 0, p->stream>>>(p->wb, p->wt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        p->wt_dirty = false;
    }
    FusedArgs f{x, y, p->wt, p->w + oB1, p->w + oB2, p->w + oB3, p->w + oB4, B, p->err};
    const int npairs = ((B + kTM - 1) / kTM + 1) / 2;
    const int grid = npairs < p->n_sm ? npairs : p->n_sm;
    mlp_fused_fwd_kernel<<<grid, kFusedThreads, kFusedSmem, p->stream>>>(f);
    return cudaGetLastError();
}

bool fused_enabled()
{
    const char *e = std::getenv("ASX_MLP_FUSED");
    return !(e && e[0] == '0');
}

bool aligned16(const void *q) { return ((uintptr_t)q & 15u) == 0; }

asx_status stage_inputs(asx_mlp *p, int B, const float *x, const float *t, int kind)
{
    const cudaMemcpyKind mk = kind == ASX_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    MLP_CUDA(p, cudaMemcpyAsync(p->xin, x, sizeof(float) * (size_t)B * kIn, mk, p->stream));
    if (t) MLP_CUDA(p, cudaMemcpyAsync(p->tin, t, sizeof(float) * (size_t)B * kOut, mk, p->stream));
    const long long n = (long long)B * kInPad;
    pad_input_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(p->xin, B, kIn, kInPad, p->x0);
    MLP_CUDA(p, cudaGetLastError());
    return ASX_OK;
}

// The two input copies of a training step into p->xin and p->tin.
asx_status copy_inputs(asx_mlp *p, int B, const float *x, const float *t, int kind)
{
    const cudaMemcpyKind mk = kind == ASX_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    MLP_CUDA(p, cudaMemcpyAsync(p->xin, x, sizeof(float) * (size_t)B * kIn, mk, p->stream));
    MLP_CUDA(p, cudaMemcpyAsync(p->tin, t, sizeof(float) * (size_t)B * kOut, mk, p->stream));
    return ASX_OK;
}

// The kernels of a training step on the inputs in p->xin / p->tin: padding, forward
// pass, gradients and the Adam update with the scalars in aa.
cudaError_t train_kernels(asx_mlp *p, int B, const AdamArgs &aa)
{
    const long long n = (long long)B * kInPad;
    pad_input_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(p->xin, B, kIn, kInPad, p->x0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = forward(p, B)) != cudaSuccess) return e;
    if ((e = backward(p, B)) != cudaSuccess) return e;
    adam_kernel<<<(unsigned)((aa.start[aa.nseg] + 255) / 256), 256, 0, p->stream>>>(aa);
    return cudaGetLastError();
}

// The graph of batch size B's step (see asx_mlp::TrainGraph), or nullptr while the step
// is to run eagerly (also for every batch size after the first kMaxTrainGraphs).
constexpr size_t kMaxTrainGraphs = 8;
asx_mlp::TrainGraph *train_graph(asx_mlp *p, int B, const AdamArgs &aa)
{
    for (auto &g : p->graphs)
        if (g.batch == B) return &g;
    if (p->graphs.size() >= kMaxTrainGraphs) return nullptr;
    if (std::find(p->seen.begin(), p->seen.end(), B) == p->seen.end()) {
        if (p->seen.size() >= 4 * kMaxTrainGraphs) return nullptr;
        p->seen.push_back(B);
        return nullptr;
    }
    asx_mlp::TrainGraph tg{B, nullptr, nullptr, nullptr, cudaKernelNodeParams{}};
    cudaGraph_t graph = nullptr;
    bool refused = true;               // some step of the capture failed
    if (p->cap || cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) == cudaSuccess) {
        const cudaStream_t user = p->stream;
        p->stream = p->cap;
        cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = train_kernels(p, B, aa);
            const cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
            if (e == cudaSuccess) e = e2;
        }
        p->stream = user;
        if (e != cudaSuccess && graph) {
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
    }
    if (graph) {
        size_t n = 0;
        std::vector<cudaGraphNode_t> nodes;
        if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess) {
            nodes.resize(n);
            if (cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) nodes.clear();
        }
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            cudaKernelNodeParams kp{};
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel &&
                cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == reinterpret_cast<void *>(adam_kernel)) {
                tg.adam = nd;
                tg.kp = kp;
            }
        }
        if (tg.adam && cudaGraphInstantiate(&tg.exec, graph, 0) != cudaSuccess) tg.exec = nullptr;
        if (tg.exec) {
            tg.graph = graph;
            refused = false;
        } else {
            cudaGraphDestroy(graph);
        }
    }
    if (refused) cudaGetLastError();   // the capture's own error is not the step's: it runs eagerly
    p->graphs.push_back(tg);
    return &p->graphs.back();
}

asx_status check_err(asx_mlp *p)
{
    int h = 0;
    MLP_CUDA(p, cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    MLP_CUDA(p, cudaStreamSynchronize(p->stream));
    if (h) return mfail(p, ASX_ETIMEOUT, "a tensor-core wait ran out");
    return ASX_OK;
}

}  // namespace

extern "C" {

asx_status asx_mlp_create(int device, void *cuda_stream, int max_batch, asx_mlp **out)
{
    if (!out || max_batch < 1 || max_batch > (1 << 22)) return ASX_EINVAL;
    *out = nullptr;
    asx_mlp *p = new (std::nothrow) asx_mlp();
    if (!p) return ASX_ENOMEM;
    p->device = device;
    p->max_batch = max_batch;
    p->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete p;
        return ASX_ECUDA;
    }
    const size_t B = (size_t)max_batch;
    const size_t nwb = (size_t)kHid * kInPad + 2 * (size_t)kHid * kHid + (size_t)kOut * kHid;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&p->w, sizeof(float) * kPadded);
    alloc((void **)&p->g, sizeof(float) * kPadded);
    alloc((void **)&p->m, sizeof(float) * kPadded);
    alloc((void **)&p->v, sizeof(float) * kPadded);
    alloc((void **)&p->wb, sizeof(__nv_bfloat16) * nwb);
    alloc((void **)&p->wt, kWtTotal);
    alloc((void **)&p->x0, sizeof(__nv_bfloat16) * B * kInPad);
    alloc((void **)&p->a1, sizeof(__nv_bfloat16) * B * kHid);
    alloc((void **)&p->a2, sizeof(__nv_bfloat16) * B * kHid);
    alloc((void **)&p->a3, sizeof(__nv_bfloat16) * B * kHid);
    alloc((void **)&p->dy, sizeof(__nv_bfloat16) * B * kOut);
    alloc((void **)&p->dz, sizeof(__nv_bfloat16) * B * kHid);
    alloc((void **)&p->dz2, sizeof(__nv_bfloat16) * B * kHid);
    alloc((void **)&p->y, sizeof(float) * B * kOut);
    alloc((void **)&p->xin, sizeof(float) * B * kIn);
    alloc((void **)&p->tin, sizeof(float) * B * kOut);
    alloc((void **)&p->loss, sizeof(float));
    alloc((void **)&p->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->w, 0, sizeof(float) * kPadded, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->m, 0, sizeof(float) * kPadded, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->v, 0, sizeof(float) * kPadded, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = refresh_bf16(p);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_fused_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        asx_mlp_destroy(p);
        return e == cudaErrorMemoryAllocation ? ASX_ENOMEM : ASX_ECUDA;
    }
    *out = p;
    return ASX_OK;
}

asx_status asx_mlp_destroy(asx_mlp *p)
{
    if (!p) return ASX_OK;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (auto &g : p->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    if (p->cap) cudaStreamDestroy(p->cap);
    void *ptrs[] = {p->w, p->g, p->m, p->v, p->wb, p->wt, p->x0, p->a1, p->a2, p->a3, p->dy, p->dz, p->dz2,
                    p->y, p->xin, p->tin, p->loss, p->err};
    for (void *q : ptrs) cudaFree(q);
    delete p;
    return ASX_OK;
}

const char *asx_mlp_last_error(const asx_mlp *p) { return p ? p->error.c_str() : "null surrogate handle"; }

asx_status asx_mlp_set_params(asx_mlp *p, const float *params, int kind)
{
    if (!p || !params) return mfail(p, ASX_EINVAL, "null argument");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return mfail(p, ASX_EINVAL, "bad ptr_kind");
    MLP_CUDA(p, cudaSetDevice(p->device));
    std::vector<float> host(ASX_MLP_PARAMS);
    if (kind == ASX_PTR_DEVICE) MLP_CUDA(p, cudaMemcpy(host.data(), params, sizeof(float) * ASX_MLP_PARAMS, cudaMemcpyDeviceToHost));
    else std::memcpy(host.data(), params, sizeof(float) * ASX_MLP_PARAMS);
    for (float f : host)
        if (!std::isfinite(f)) return mfail(p, ASX_EINVAL, "non-finite parameter");
    std::vector<float> pad;
    pack_to_padded(host.data(), pad);
    MLP_CUDA(p, cudaMemcpyAsync(p->w, pad.data(), sizeof(float) * kPadded, cudaMemcpyHostToDevice, p->stream));
    MLP_CUDA(p, cudaMemsetAsync(p->m, 0, sizeof(float) * kPadded, p->stream));
    MLP_CUDA(p, cudaMemsetAsync(p->v, 0, sizeof(float) * kPadded, p->stream));
    MLP_CUDA(p, refresh_bf16(p));
    p->wt_dirty = true;
    MLP_CUDA(p, cudaStreamSynchronize(p->stream));
    p->adam_t = 0;
    return ASX_OK;
}

asx_status asx_mlp_get_params(asx_mlp *p, float *params, int kind)
{
    if (!p || !params) return mfail(p, ASX_EINVAL, "null argument");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return mfail(p, ASX_EINVAL, "bad ptr_kind");
    MLP_CUDA(p, cudaSetDevice(p->device));
    std::vector<float> pad(kPadded), host(ASX_MLP_PARAMS);
    MLP_CUDA(p, cudaMemcpyAsync(pad.data(), p->w, sizeof(float) * kPadded, cudaMemcpyDeviceToHost, p->stream));
    MLP_CUDA(p, cudaStreamSynchronize(p->stream));
    padded_to_pack(pad, host.data());
    if (kind == ASX_PTR_DEVICE) MLP_CUDA(p, cudaMemcpy(params, host.data(), sizeof(float) * ASX_MLP_PARAMS, cudaMemcpyHostToDevice));
    else std::memcpy(params, host.data(), sizeof(float) * ASX_MLP_PARAMS);
    return ASX_OK;
}

asx_status asx_mlp_forward(asx_mlp *p, int batch, const float *x, float *y, int kind)
{
    if (!p || !x || !y) return mfail(p, ASX_EINVAL, "null argument");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return mfail(p, ASX_EINVAL, "bad ptr_kind");
    MLP_CUDA(p, cudaSetDevice(p->device));
    const cudaMemcpyKind back = kind == ASX_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (batch < 1) return batch == 0 ? ASX_OK : mfail(p, ASX_EINVAL, "negative batch");
    if (fused_enabled()) {
        if (kind == ASX_PTR_DEVICE && aligned16(x) && aligned16(y)) {
            MLP_CUDA(p, fused_forward(p, batch, x, y));      // the whole batch in one launch
            return ASX_OK;
        }
        const cudaMemcpyKind in = kind == ASX_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        for (int b0 = 0; b0 < batch; b0 += p->max_batch) {
            const int B = batch - b0 < p->max_batch ? batch - b0 : p->max_batch;
            MLP_CUDA(p, cudaMemcpyAsync(p->xin, x + (size_t)b0 * kIn, sizeof(float) * (size_t)B * kIn, in, p->stream));
            MLP_CUDA(p, fused_forward(p, B, p->xin, p->y));
            MLP_CUDA(p, cudaMemcpyAsync(y + (size_t)b0 * kOut, p->y, sizeof(float) * (size_t)B * kOut, back, p->stream));
        }
        if (kind == ASX_PTR_HOST) return check_err(p);
        return ASX_OK;
    }
    for (int b0 = 0; b0 < batch; b0 += p->max_batch) {
        const int B = batch - b0 < p->max_batch ? batch - b0 : p->max_batch;
        asx_status st = stage_inputs(p, B, x + (size_t)b0 * kIn, nullptr, kind);
        if (st) return st;
        MLP_CUDA(p, forward(p, B));
        MLP_CUDA(p, cudaMemcpyAsync(y + (size_t)b0 * kOut, p->y, sizeof(float) * (size_t)B * kOut, back, p->stream));
    }
    if (kind == ASX_PTR_HOST) return check_err(p);
    return ASX_OK;
}

asx_status asx_mlp_gradients(asx_mlp *p, int batch, const float *x, const float *t, float *grad, float *loss,
                             int kind)
{
    if (!p || !x || !t || !grad) return mfail(p, ASX_EINVAL, "null argument");
    if (batch < 1 || batch > p->max_batch) return mfail(p, ASX_EINVAL, "batch out of range");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return mfail(p, ASX_EINVAL, "bad ptr_kind");
    MLP_CUDA(p, cudaSetDevice(p->device));
    asx_status st = stage_inputs(p, batch, x, t, kind);
    if (st) return st;
    MLP_CUDA(p, forward(p, batch));
    MLP_CUDA(p, backward(p, batch));
    std::vector<float> pad(kPadded), host(ASX_MLP_PARAMS);
    float l = 0.0f;
    MLP_CUDA(p, cudaMemcpyAsync(pad.data(), p->g, sizeof(float) * kPadded, cudaMemcpyDeviceToHost, p->stream));
    MLP_CUDA(p, cudaMemcpyAsync(&l, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    st = check_err(p);
    if (st) return st;
    padded_to_pack(pad, host.data());
    if (kind == ASX_PTR_DEVICE) MLP_CUDA(p, cudaMemcpy(grad, host.data(), sizeof(float) * ASX_MLP_PARAMS, cudaMemcpyHostToDevice));
    else std::memcpy(grad, host.data(), sizeof(float) * ASX_MLP_PARAMS);
    if (loss) *loss = l;
    return ASX_OK;
}

asx_status asx_mlp_train_step(asx_mlp *p, int batch, const float *x, const float *t, float lr, float weight_decay,
                              float *loss, int kind)
{
    if (!p || !x || !t) return mfail(p, ASX_EINVAL, "null argument");
    if (batch < 1 || batch > p->max_batch) return mfail(p, ASX_EINVAL, "batch out of range");
    if (!(lr > 0.0f) || !(weight_decay >= 0.0f)) return mfail(p, ASX_EINVAL, "bad learning rate");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return mfail(p, ASX_EINVAL, "bad ptr_kind");
    MLP_CUDA(p, cudaSetDevice(p->device));
    asx_status st = copy_inputs(p, batch, x, t, kind);
    if (st) return st;
    p->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow((double)b1, (double)p->adam_t);
    const float c2 = 1.0f - (float)std::pow((double)b2, (double)p->adam_t);
    // weights (with BF16 copies) and biases (FP32 only, no decay)
    const long long segs[8][3] = {{oW1, (long long)kHid * kInPad, 0}, {oB1, kHid, -1}, {oW2, (long long)kHid * kHid, 1},
                                  {oB2, kHid, -1}, {oW3, (long long)kHid * kHid, 2}, {oB3, kHid, -1},
                                  {oW4, (long long)kOut * kHid, 3}, {oB4, kOut, -1}};
    AdamArgs aa{};
    aa.nseg = 8;
    aa.lr = lr;
    aa.b1 = b1;
    aa.b2 = b2;
    aa.eps = 1e-8f;
    aa.c1 = c1;
    aa.c2 = c2;
    for (int s = 0; s < 8; s++) {
        const long long o = segs[s][0], n = segs[s][1];
        const int l = (int)segs[s][2];
        aa.w[s] = p->w + o;
        aa.grad[s] = p->g + o;
        aa.mo[s] = p->m + o;
        aa.ve[s] = p->v + o;
        aa.wb[s] = l >= 0 ? wb_of(p, l) : nullptr;
        aa.wd[s] = l >= 0 ? weight_decay : 0.0f;
        aa.start[s + 1] = aa.start[s] + (int)n;
    }
    asx_mlp::TrainGraph *tg = train_graph(p, batch, aa);
    if (tg && tg->exec) {
        void *args[] = {(void *)&aa};
        cudaKernelNodeParams kp = tg->kp;
        kp.kernelParams = args;
        kp.extra = nullptr;
        MLP_CUDA(p, cudaGraphExecKernelNodeSetParams(tg->exec, tg->adam, &kp));
        MLP_CUDA(p, cudaGraphLaunch(tg->exec, p->stream));
    } else {
        MLP_CUDA(p, train_kernels(p, batch, aa));
    }
    p->wt_dirty = true;
    if (loss) {
        MLP_CUDA(p, cudaMemcpyAsync(loss, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
        return check_err(p);
    }
    return ASX_OK;
}

asx_status asx_surrogate_check(int batch, int n_check, const int *idx, float *y, const float *ref, float tol,
                               float *rel_err, int *n_replaced, void *cuda_stream)
{
    if (batch < 0 || n_check < 0 || n_check > batch || !(tol >= 0.0f)) return ASX_EINVAL;
    if (n_check > 0 && (!idx || !y || !ref || !rel_err || !n_replaced)) return ASX_EINVAL;
    if (!n_replaced) return ASX_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(n_replaced, 0, sizeof(int), st) != cudaSuccess) return ASX_ECUDA;
    if (n_check == 0) return ASX_OK;
    const unsigned blocks = (unsigned)(((long long)n_check * 32 + 255) / 256);
    asx::hydro_check_kernel<<<blocks, 256, 0, st>>>(batch, n_check, kOut, idx, y, ref, tol, rel_err, n_replaced);
    return cudaGetLastError() == cudaSuccess ? ASX_OK : ASX_ECUDA;
}

}  // extern "C"
