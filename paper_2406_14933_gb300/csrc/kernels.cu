// kernels.cu -- device code of the hexagonal porous Saint-Venant step (sm_103a).
//
// One time step of the explicit finite-volume scheme (Sec. 2.2, Eq. fvm_2D_eq_frac.07,
// split as in Appendix A):
//   * per edge (i, j): interface velocity and normal component (Eq. fvm_2D_eq.04),
//     upwind mass (Eq. fvm_2D_eq.06), pressure-term mass (Eq. fvm_2D_eq.05), and the
//     edge terms of the operators L, J, S (Eq. fvm_2D_eq_frac.01);
//   * per cell: transport of theta*h and theta*h*v (Eqs. fvm_2D_eq_frac.05-1/-2), rain
//     at t^{n+1} (Eq. fvm_2D_eq_frac.06-1), closed-form implicit friction
//     (Eq. fvm_2D_eq_frac.06-2 via Eq. miu-formula), wave speed for the next CFL step
//     (Eq. fvm_2D_eq_frac.13);
//   * per step: max wave speed, boundary outflow, clamped water (CTA partials and
//     atomics), then the last CTA books the ledger, advances the clock and prepares
//     the next step's dt (Eq. fvm_2D_eq_frac.12) on the device.
//
// Precision: state in float32; the mass theta*h is a compensated pair hi + lo, and
// every mass increment is added with an error-free two-sum so the water budget closes
// to float64 rounding.  Each edge's mass increment is evaluated once per edge in a
// canonical orientation (lower cell index first) with explicitly rounded operations,
// so both cells of an edge apply bit-identical, opposite increments.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "device_common.cuh"

namespace asx {

namespace {

// ------------------------------------------------------------ step: gather variant

constexpr int kGX = 32, kGY = 8;

// One thread per cell: loads the cell and its six neighbours, evaluates the six edges
// (each in the canonical orientation, so a shared edge gives both cells the same
// increment), updates the cell and writes the other state buffer.
__global__ void __launch_bounds__(kGX *kGY) step_gather_kernel(const StepArgs a)
{
    const DevCtl *ctl = a.ctl;
    if (!ctl->active) return;
    const StepScalars sc = step_scalars(a);
    const int c = blockIdx.x * kGX + threadIdx.x;
    const int r = blockIdx.y * kGY + threadIdx.y;
    unsigned cb = 0u;
    FF outd, clq;
    if (r < a.rows && c < a.cols) gather_cell(a, sc, r, c, cb, outd, clq);
    reduce_and_finish<kGX * kGY>(a, cb, outd.value(), clq.value());
}

// --------------------------------------------------------------- control kernels

__global__ void prepare_kernel(DevCtl *c, int mode, double t_end, long long n_steps)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == kPrepSteps) {
        c->t_end = INFINITY;
        c->step_limit = c->step + n_steps;
    } else if (mode == kPrepUntil) {
        c->t_end = t_end;
        c->step_limit = 0x7fffffffffffffffLL;
    }
    prepare_step(c);
}

constexpr int kScanThreads = 256;

// Storage sum_i sigma (hi + lo) in float64 and c_max of the current state.  Block
// partials, then the last block sums them in a fixed order (deterministic).
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const StepArgs a, double *parts,
                                                            int set_storage0)
{
    DevCtl *ctl = a.ctl;
    const int par = ctl->parity;
    const float *mhi = a.mhi[par], *mlo = a.mlo[par], *v1 = a.v1[par], *v2 = a.v2[par];
    const long long n = (long long)a.rows * a.cols;
    double s = 0.0;
    unsigned cmb = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const float hi = mhi[k];
        s += (double)hi + (double)mlo[k];
        const float h = __fmul_rn(hi, cell_rtheta(a, k));
        cmb = max(cmb, speed_bits(wave_speed(v1[k], v2[k], h, a.g)));
    }
    __shared__ double ss[kScanThreads / 32];
    __shared__ unsigned sm[kScanThreads / 32];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    unsigned bits = __reduce_max_sync(0xffffffffu, cmb);
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = bits;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        unsigned bm = 0u;
        for (int w = 0; w < kScanThreads / 32; w++) {
            bs += ss[w];
            bm = max(bm, sm[w]);
        }
        parts[2 * blockIdx.x] = bs;
        parts[2 * blockIdx.x + 1] = (double)__uint_as_float(bm);
        __threadfence();
        last = atomicAdd(&ctl->scan_done, 1u) == gridDim.x - 1;
        if (last) {
            __threadfence();
            volatile double *vp = parts;
            double tot = 0.0;
            unsigned cmx = 0u;
            for (unsigned b = 0; b < gridDim.x; b++) {
                tot += vp[2 * b];
                cmx = max(cmx, speed_bits((float)vp[2 * b + 1]));
            }
            ctl->storage = tot * ctl->sigma;
            if (set_storage0) ctl->storage0 = ctl->storage;
            ctl->cmax_cur = __uint_as_float(cmx);
            if (!(ctl->cmax_cur <= FLT_MAX)) ctl->err |= kErrNumeric;
            ctl->scan_done = 0u;
        }
    }
}

// theta*h in float64 (exact product of two floats), split into hi + lo; velocities.
// h, v1, v2 are pitched device buffers (v1, v2 may be nullptr = 0).
__global__ void init_state_kernel(const StepArgs a, int par, const float *h, const float *v1,
                                  const float *v2)
{
    const long long n = (long long)a.rows * a.cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double m = (double)cell_theta(a, k) * (double)h[k];
        const float hi = (float)m;
        const float lo = (float)(m - (double)hi);
        const float u1 = v1 ? v1[k] : 0.0f, u2 = v2 ? v2[k] : 0.0f;
        a.mhi[par][k] = hi;
        a.mlo[par][k] = lo;
        a.v1[par][k] = u1;
        a.v2[par][k] = u2;
    }
}

// Depth h = (hi + lo) / theta into a pitched float32 buffer.
__global__ void extract_depth_kernel(const StepArgs a, int par, float *hout)
{
    const long long n = (long long)a.rows * a.cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double m = (double)a.mhi[par][k] + (double)a.mlo[par][k];
        hout[k] = (float)(m / (double)cell_theta(a, k));
    }
}

int elementwise_blocks(int rows, int cols)
{
    const long long n = (long long)rows * cols;
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ------------------------------------------------------------------- launchers

int step_gather_blocks(int rows, int cols)
{
    return ((cols + kGX - 1) / kGX) * ((rows + kGY - 1) / kGY);
}

cudaError_t launch_step_gather(const StepArgs &a, cudaStream_t s)
{
    dim3 grid((a.cols + kGX - 1) / kGX, (a.rows + kGY - 1) / kGY);
    step_gather_kernel<<<grid, dim3(kGX, kGY), 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prepare(DevCtl *ctl, int mode, double t_end, long long n_steps, cudaStream_t s)
{
    prepare_kernel<<<1, 32, 0, s>>>(ctl, mode, t_end, n_steps);
    return cudaGetLastError();
}

int scan_blocks(int rows, int cols) { return elementwise_blocks(rows, cols); }

cudaError_t launch_scan(const StepArgs &a, double *partials, int nparts, int set_storage0,
                        cudaStream_t s)
{
    scan_kernel<<<nparts, kScanThreads, 0, s>>>(a, partials, set_storage0);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const StepArgs &a, int parity, const float *h, const float *v1,
                              const float *v2, cudaStream_t s)
{
    init_state_kernel<<<elementwise_blocks(a.rows, a.cols), 256, 0, s>>>(a, parity, h, v1, v2);
    return cudaGetLastError();
}

cudaError_t launch_extract_depth(const StepArgs &a, int parity, float *h_out, cudaStream_t s)
{
    extract_depth_kernel<<<elementwise_blocks(a.rows, a.cols), 256, 0, s>>>(a, parity, h_out);
    return cudaGetLastError();
}

}  // namespace asx
