// step_strip.cu -- the main step kernel: one-warp CTAs, each a strip tile worker
// (strip_tile.cuh) over one 128-column tile of the raster, or a frame CTA gathering the
// cells along the raster's sides; the last CTA finishes the step.
#include "strip_tile.cuh"

namespace asx {

namespace {

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

namespace {

// One warp waits, with the step kernels' bounded wait, on an mbarrier nothing arrives at,
// and flags the timeout.
__global__ void wait_selftest_kernel(int *err)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u)) atomicOr(err, kErrTimeout);
}

}  // namespace

}  // namespace asx

extern "C" asx_status asx_selftest_wait(int device)
{
    if (cudaSetDevice(device) != cudaSuccess) return ASX_ECUDA;
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return ASX_ENOMEM;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        asx::wait_selftest_kernel<<<1, 32>>>(err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return ASX_ECUDA;
    return (h & asx::kErrTimeout) ? ASX_ETIMEOUT : ASX_OK;
}
