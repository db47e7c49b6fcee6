// noalloc.cu -- the allocation-free entry point asx_state_scan_noalloc.
//
// Some callers cannot allocate device memory at all: an embedding runtime that owns
// every buffer and forbids allocation after start-up, a process inside a memory pool
// that is already full, or a tool that only holds pointers lent to it by another
// library.  For them this file offers the water-storage / wave-speed scan of a state
// they already hold, with its scratch (one partial per CTA and a completion counter) in
// a fixed file-scope device array instead of memory obtained from cudaMalloc.
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "device_common.cuh"

namespace asx {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocCellsPerBlock = kNoAllocThreads * 64;   // cells one CTA sums
constexpr int kNoAllocMaxBlocks = 4096;                      // partials the scratch holds
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: per-CTA partial sums (float64 storage and
// the wave-speed bits), then the completion counter.  64 KB + 256 bytes per device.
struct NoAllocScratch {
    double storage[kNoAllocMaxBlocks];
    unsigned cmax_bits[kNoAllocMaxBlocks];
    unsigned done;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(kNoAllocThreads)
scan_noalloc_kernel(NoAllocScratch *sc, int rows, int cols, int pitch, const float *mhi,
                    const float *mlo, const float *v1, const float *v2, const float *theta,
                    float g, double sigma, double *storage_out, float *cmax_out)
{
    const long long n = (long long)rows * cols;
    const long long b0 = (long long)blockIdx.x * kNoAllocCellsPerBlock;
    const long long b1 = min(n, b0 + kNoAllocCellsPerBlock);
    double s = 0.0;
    unsigned cmb = 0u;
    for (long long i = b0 + threadIdx.x; i < b1; i += kNoAllocThreads) {
        const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
        const size_t k = (size_t)r * pitch + c;
        const float hi = mhi[k];
        s += (double)hi + (double)mlo[k];
        const float h = __fmul_rn(hi, fast_rcp(theta[k]));
        cmb = max(cmb, speed_bits(wave_speed(v1[k], v2[k], h, g)));
    }
    __shared__ double ss[kNoAllocThreads / 32];
    __shared__ unsigned sm[kNoAllocThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const unsigned bits = __reduce_max_sync(0xffffffffu, cmb);
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = bits;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        unsigned bm = 0u;
        for (int w = 0; w < kNoAllocThreads / 32; w++) {
            bs += ss[w];
            bm = max(bm, sm[w]);
        }
        sc->storage[blockIdx.x] = bs;
        sc->cmax_bits[blockIdx.x] = bm;
        __threadfence();
        if (atomicAdd(&sc->done, 1u) == gridDim.x - 1) {
            // last CTA: fixed-order sum of the partials, then clear the counter
            __threadfence();
            const volatile double *vs = sc->storage;
            const volatile unsigned *vm = sc->cmax_bits;
            double tot = 0.0;
            unsigned cm = 0u;
            for (unsigned b = 0; b < gridDim.x; b++) {
                tot += vs[b];
                cm = max(cm, vm[b]);
            }
            *storage_out = tot * sigma;
            *cmax_out = __uint_as_float(cm);
            sc->done = 0u;
        }
    }
}

// Device address of the scratch array, looked up once per device (host code may not use
// the symbol itself as an address).  Atomic slots: threads making their first call on
// the same device at once each look the address up and store the same value.
std::atomic<NoAllocScratch *> g_scratch_addr[kMaxDevices];

}  // namespace
}  // namespace asx

using namespace asx;

extern "C" asx_status asx_state_scan_noalloc(int rows, int cols, int pitch, double edge_m, double g,
                                             const float *m_hi, const float *m_lo, const float *v1,
                                             const float *v2, const float *theta, double *storage_out,
                                             float *cmax_out, void *cuda_stream)
{
    if (rows < 1 || cols < 1 || pitch < cols || !(edge_m > 0.0) || !std::isfinite(edge_m) || !(g > 0.0) ||
        !std::isfinite(g))
        return ASX_EINVAL;
    if (!m_hi || !m_lo || !v1 || !v2 || !theta || !storage_out || !cmax_out) return ASX_EINVAL;
    const long long n = (long long)rows * cols;
    const long long nblocks = (n + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock;
    if (nblocks > kNoAllocMaxBlocks) return ASX_EINVAL;     // more than 67,108,864 cells
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ASX_ECUDA;
    NoAllocScratch *sc = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!sc) {
        // first call on this device: find the device address of the scratch array
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ASX_ECUDA;
        sc = static_cast<NoAllocScratch *>(p);
        g_scratch_addr[dev].store(sc, std::memory_order_release);
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the counter must start at zero even if an earlier call was cut short
    if (cudaMemsetAsync(&sc->done, 0, sizeof(unsigned), s) != cudaSuccess) return ASX_ECUDA;
    const double sigma = 1.5 * std::sqrt(3.0) * edge_m * edge_m;
    const float gf = (float)g;
    // cudaLaunchKernel returns this launch's own status: a launch error that earlier,
    // unrelated work left for cudaGetLastError is neither reported nor cleared here
    void *args[] = {&sc, &rows, &cols, &pitch, (void *)&m_hi, (void *)&m_lo, (void *)&v1, (void *)&v2,
                    (void *)&theta, (void *)&gf, (void *)&sigma, &storage_out, &cmax_out};
    const cudaError_t e = cudaLaunchKernel((const void *)scan_noalloc_kernel, dim3((unsigned)nblocks),
                                           dim3(kNoAllocThreads), args, 0, s);
    return e == cudaSuccess ? ASX_OK : ASX_ECUDA;
}
