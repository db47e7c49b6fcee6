// step_fp64.cu -- the double-precision mode of the step (asx_raster_desc.precision =
// ASX_FP64): the same scheme as the float32 kernels (Sec. 2.2, Eq. fvm_2D_eq_frac.07 in
// the fractional form of Appendix A) with the state, the bed, the porosity and every
// operation in float64.
//
// One thread per cell gathers its six neighbours and sums each operator over them from
// the cell's own side, in the direction order E, NE, NW, W, SW, SE: the interface
// velocity and its normal component (Eq. fvm_2D_eq.04), the upwind mass (Eq.
// fvm_2D_eq.06), the pressure-term mass with its tie rule (Eq. fvm_2D_eq.05), then L, J
// and S (Eq. fvm_2D_eq_frac.01); the boundary sides as ghost cells (wall, free
// discharge, given mass flux, Dirichlet).  A flux seen from the other cell is the exact
// negative (the interface velocity is a commutative sum, the normal is negated), so
// mass moves antisymmetrically.  The cell update takes the transport, the rain at
// t^{n+1} and the closed-form implicit friction (Eq. miu-formula).  The file is built
// without contraction of multiplies and adds into fused multiply-adds, so every
// operation rounds as written.  GB300 runs float64 at 1/64 of its float32 rate: this
// mode serves checks against double-precision references on small rasters, not speed.
#include <cfloat>
#include <cmath>

#include "device_common.cuh"

namespace asx {

namespace {

constexpr int kFX = 32, kFY = 8;
constexpr double kS32d = 0.86602540378443864676;   // sqrt(3) / 2

__device__ __forceinline__ void normal64(int d, double &n1, double &n2)
{
    switch (d) {
    case 0: n1 = 1.0; n2 = 0.0; break;
    case 1: n1 = 0.5; n2 = kS32d; break;
    case 2: n1 = -0.5; n2 = kS32d; break;
    case 3: n1 = -1.0; n2 = 0.0; break;
    case 4: n1 = -0.5; n2 = -kS32d; break;
    default: n1 = 0.5; n2 = -kS32d; break;
    }
}

__device__ __forceinline__ double theta64(const StepArgs64 &a, size_t k)
{
    return a.cls ? a.cls_theta[a.cls[k]] : a.theta[k];
}

__device__ __forceinline__ int side_type64(const StepArgs64 &a, int side, int pos)
{
    if (a.fb[side] == a.fe[side]) return a.bc[side];
    return (pos >= a.fb[side] && pos < a.fe[side]) ? a.bc[side] : ASX_BC_WALL;
}

__device__ __forceinline__ double speed64(double v1, double v2, double h, double g)
{
    return sqrt(v1 * v1 + v2 * v2) + sqrt(g * h);
}

// The step for cell (r, c): writes the new state of the other parity and returns the
// new wave speed, the cell's boundary mass increment (outflow positive) and its clamped
// mass, both per unit area.
__device__ void cell64(const StepArgs64 &a, int par, double dt, double qr, int r, int c, double &cnew,
                       double &outd, double &clampd)
{
    const double *m = a.m[par], *w1 = a.v1[par], *w2 = a.v2[par];
    const size_t k = (size_t)r * a.pitch + c;
    const double l = a.l, g = a.g;
    const double mi = m[k], ui = w1[k], wi = w2[k], zi = a.z[k], thi = theta64(a, k);
    const double hi = mi / thi;
    double L = 0.0, J1 = 0.0, J2 = 0.0, S1 = 0.0, S2 = 0.0, out_rate = 0.0;
    double ci = 0.0;
    if (a.visc) ci = speed64(ui, wi, hi, g);
    for (int d = 0; d < 6; d++) {
        double n1, n2;
        normal64(d, n1, n2);
        int rr, cc, side;
        if (neighbour(a.rows, a.cols, r, c, d, rr, cc, side)) {
            const size_t j = (size_t)rr * a.pitch + cc;
            const double mj = m[j], uj = w1[j], wj = w2[j];
            const double hj = mj / theta64(a, j);
            const double vb1 = (ui + uj) / 2.0, vb2 = (wi + wj) / 2.0;
            const double vn = vb1 * n1 + vb2 * n2;
            const double dw = g * ((a.z[j] - zi) + (hj - hi));
            double up = 0.0;
            if (vn > 0.0) up = mi;
            else if (vn < 0.0) up = mj;
            const double hat = vn != 0.0 ? up : (dw < 0.0 ? mi : mj);
            L -= l * up * vn;
            J1 -= l * up * vb1 * vn;
            J2 -= l * up * vb2 * vn;
            S1 -= 0.5 * l * dw * hat * n1;
            S2 -= 0.5 * l * dw * hat * n2;
            if (a.visc) {
                const double cj = speed64(uj, wj, hj, g);
                const double cij = ci > cj ? ci : cj;
                const double den = mi + mj;
                const double mu = den > 0.0 ? 2.0 * mi * mj / den : 0.0;
                J1 += l * cij * mu * (uj - ui);
                J2 += l * cij * mu * (wj - wi);
            }
        } else {
            const int bt = side_type64(a, side, (side == ASX_SIDE_S || side == ASX_SIDE_N) ? c : r);
            const double ns1 = side == ASX_SIDE_W ? -1.0 : side == ASX_SIDE_E ? 1.0 : 0.0;
            const double ns2 = side == ASX_SIDE_S ? -1.0 : side == ASX_SIDE_N ? 1.0 : 0.0;
            if (bt == ASX_BC_FREE) {
                // ghost copy of the cell: outflow only, no pressure term
                const double vn = ui * n1 + wi * n2;
                if (vn > 0.0) {
                    L -= l * mi * vn;
                    J1 -= l * mi * ui * vn;
                    J2 -= l * mi * wi * vn;
                    out_rate += l * mi * vn;
                }
            } else if (bt == ASX_BC_FLUX && a.bq[side] > 0.0) {
                // given mass flux q along the inward normal, at the cell's depth but no
                // shallower than the critical depth; no pressure term
                const double q = a.bq[side];
                const double qin = l * q * (ns1 * n1 + ns2 * n2);
                const double hc = cbrt(q * q / g);
                const double uin = q / (hi > hc ? hi : hc);
                L += qin;
                J1 += qin * uin * (-ns1);
                J2 += qin * uin * (-ns2);
                out_rate -= qin;
            } else if (bt == ASX_BC_DIRICHLET) {
                // ghost on the cell's bed and porosity with the side's depth and inflow
                const double hg = a.bh[side], mg = thi * hg;
                const double ug = -a.bu[side] * ns1, wg = -a.bu[side] * ns2;
                const double vb1 = (ui + ug) / 2.0, vb2 = (wi + wg) / 2.0;
                const double vn = vb1 * n1 + vb2 * n2;
                const double dw = g * (hg - hi);
                double up = 0.0;
                if (vn > 0.0) up = mi;
                else if (vn < 0.0) up = mg;
                const double hat = vn != 0.0 ? up : (dw < 0.0 ? mi : mg);
                L -= l * up * vn;
                J1 -= l * up * vb1 * vn;
                J2 -= l * up * vb2 * vn;
                S1 -= 0.5 * l * dw * hat * n1;
                S2 -= 0.5 * l * dw * hat * n2;
                out_rate += l * up * vn;
            }
            // wall: mirror ghost, nothing crosses
        }
    }
    const double kap = dt / (1.5 * sqrt(3.0) * l * l);
    // transport of theta h, rain at t^{n+1}, transport of theta h v with the surface force
    double mnew = mi + kap * L;
    mnew = mnew + qr;
    const double g1 = mi * ui + kap * (J1 + S1);
    const double g2 = mi * wi + kap * (J2 + S2);
    clampd = 0.0;
    if (mnew < 0.0) {
        clampd = -mnew;
        mnew = 0.0;
    }
    // implicit resistance: alpha v + beta |v| v = gamma, alpha = theta h (+ dt tau h),
    // beta = dt K(h, theta), K = alpha_p h (1 - theta) + theta alpha_s
    const double hn = mnew / thi;
    double as, ap;
    if (a.cls) {
        as = a.cls_as[a.cls[k]];
        ap = a.cls_ap[a.cls[k]];
    } else {
        as = a.alpha_s;
        ap = a.alpha_p;
    }
    const double beta = dt * (ap * hn * (1.0 - thi) + thi * as);
    const double alpha = mnew + dt * a.tau * hn;
    const double ng = hypot(g1, g2);
    const double den = alpha + sqrt(alpha * alpha + 4.0 * beta * ng);
    double v1n = 0.0, v2n = 0.0;
    if (den > 0.0) {
        v1n = 2.0 * g1 / den;
        v2n = 2.0 * g2 / den;
    }
    if (hn < a.h_dry) {
        v1n = 0.0;
        v2n = 0.0;
    }
    const int np = par ^ 1;
    a.m[np][k] = mnew;
    a.v1[np][k] = v1n;
    a.v2[np][k] = v2n;
    cnew = speed64(v1n, v2n, hn, g);
    outd = kap * out_rate;
}

__device__ __forceinline__ unsigned long long shfl_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block reduction (largest wave speed as the bits of a non-negative double, which order
// like the values; NaN sorts above +Inf), order-independent ledger sums, last-CTA finish.
template <int NT>
__device__ void reduce_finish64(const StepArgs64 &a, unsigned long long cb, double outq, double clq)
{
    __shared__ unsigned long long s_max[NT / 32];
    __shared__ double s_out[NT / 32], s_cl[NT / 32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    cb = shfl_max_u64(cb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        outq += __shfl_down_sync(0xffffffffu, outq, o);
        clq += __shfl_down_sync(0xffffffffu, clq, o);
    }
    if (lane == 0) {
        s_max[wid] = cb;
        s_out[wid] = outq;
        s_cl[wid] = clq;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long mb = 0ull;
        double so = 0.0, sc = 0.0;
        for (int w = 0; w < NT / 32; w++) {
            mb = s_max[w] > mb ? s_max[w] : mb;
            so += s_out[w];
            sc += s_cl[w];
        }
        DevCtl *ctl = a.ctl;
        atomicMax(&ctl->cmax64_bits, mb);
        if (so != 0.0) fx_add(ctl->out_fx, so);
        if (sc != 0.0) fx_add(ctl->clamp_fx, sc);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->done_ctas, 1u);
        if (prev == (unsigned)a.nblocks - 1u) {
            __threadfence();
            finish_step(ctl);
        }
    }
}

__global__ void __launch_bounds__(kFX *kFY) step_fp64_kernel(const StepArgs64 a)
{
    const DevCtl *ctl = a.ctl;
    if (!ctl->active) return;
    const int par = ctl->parity;
    const double dt = ctl->dt, qr = ctl->qr64;
    const int c = blockIdx.x * kFX + threadIdx.x;
    const int r = blockIdx.y * kFY + threadIdx.y;
    unsigned long long cb = 0ull;
    double outd = 0.0, cld = 0.0;
    if (r < a.rows && c < a.cols) {
        double cn;
        cell64(a, par, dt, qr, r, c, cn, outd, cld);
        cb = (unsigned long long)__double_as_longlong(cn);
    }
    reduce_finish64<kFX * kFY>(a, cb, outd, cld);
}

constexpr int kScan64Threads = 256;

// Storage sum_i sigma m_i and the largest wave speed of the current state; block
// partials summed in a fixed order by the last block.
__global__ void __launch_bounds__(kScan64Threads) scan64_kernel(const StepArgs64 a, double *parts, int set_storage0)
{
    DevCtl *ctl = a.ctl;
    const int par = ctl->parity;
    const long long n = (long long)a.rows * a.cols;
    double s = 0.0;
    unsigned long long cb = 0ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double m = a.m[par][k];
        s += m;
        const double sp = speed64(a.v1[par][k], a.v2[par][k], m / theta64(a, k), a.g);
        const unsigned long long b = (unsigned long long)__double_as_longlong(sp);
        cb = b > cb ? b : cb;
    }
    __shared__ double ss[kScan64Threads / 32];
    __shared__ unsigned long long sm[kScan64Threads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    cb = shfl_max_u64(cb);
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = cb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        unsigned long long bm = 0ull;
        for (int w = 0; w < kScan64Threads / 32; w++) {
            bs += ss[w];
            bm = sm[w] > bm ? sm[w] : bm;
        }
        parts[2 * blockIdx.x] = bs;
        parts[2 * blockIdx.x + 1] = __longlong_as_double((long long)bm);
        __threadfence();
        if (atomicAdd(&ctl->scan_done, 1u) == gridDim.x - 1) {
            __threadfence();
            const volatile double *vp = parts;
            double tot = 0.0;
            unsigned long long cmx = 0ull;
            for (unsigned b = 0; b < gridDim.x; b++) {
                tot += vp[2 * b];
                const unsigned long long x = (unsigned long long)__double_as_longlong(vp[2 * b + 1]);
                cmx = x > cmx ? x : cmx;
            }
            ctl->storage = tot * ctl->sigma;
            if (set_storage0) ctl->storage0 = ctl->storage;
            ctl->cmax64_cur = __longlong_as_double((long long)cmx);
            if (!(ctl->cmax64_cur <= DBL_MAX)) ctl->err |= kErrNumeric;
            ctl->scan_done = 0u;
        }
    }
}

__global__ void init64_kernel(const StepArgs64 a, int par, const float *h, const float *v1, const float *v2)
{
    const long long n = (long long)a.rows * a.cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double hk = (double)h[k];
        const double u1 = v1 ? (double)v1[k] : 0.0, u2 = v2 ? (double)v2[k] : 0.0;
        a.m[par][k] = theta64(a, k) * hk;
        a.v1[par][k] = u1;
        a.v2[par][k] = u2;
    }
}

__global__ void extract64_kernel(const StepArgs64 a, int par, double *h64, double *v164, double *v264, float *h32,
                                 float *v132, float *v232)
{
    const long long n = (long long)a.rows * a.cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double h = a.m[par][k] / theta64(a, k);
        if (h64) h64[k] = h;
        if (v164) v164[k] = a.v1[par][k];
        if (v264) v264[k] = a.v2[par][k];
        if (h32) h32[k] = (float)h;
        if (v132) v132[k] = (float)a.v1[par][k];
        if (v232) v232[k] = (float)a.v2[par][k];
    }
}

__global__ void extract_wide_kernel(const StepArgs a, int par, double *h, double *v1, double *v2)
{
    const long long n = (long long)a.rows * a.cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const double th = a.cls ? (double)a.cls_theta[a.cls[k]] : (double)a.theta[k];
        if (h) h[k] = ((double)a.mhi[par][k] + (double)a.mlo[par][k]) / th;
        if (v1) v1[k] = (double)a.v1[par][k];
        if (v2) v2[k] = (double)a.v2[par][k];
    }
}

__global__ void narrow_kernel(const double *src, int rows, int cols, int sp, float *dst, int dp)
{
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
        dst[(size_t)r * dp + c] = (float)src[(size_t)r * sp + c];
    }
}

__global__ void widen_kernel(const float *src, int rows, int cols, int sp, double *dst, int dp)
{
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
        dst[(size_t)r * dp + c] = (double)src[(size_t)r * sp + c];
    }
}

int blocks_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int step_fp64_blocks(int rows, int cols) { return ((cols + kFX - 1) / kFX) * ((rows + kFY - 1) / kFY); }

cudaError_t launch_step_fp64(const StepArgs64 &a, cudaStream_t s)
{
    dim3 grid((a.cols + kFX - 1) / kFX, (a.rows + kFY - 1) / kFY);
    step_fp64_kernel<<<grid, dim3(kFX, kFY), 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan64(const StepArgs64 &a, double *partials, int nparts, int set_storage0, cudaStream_t s)
{
    scan64_kernel<<<nparts, kScan64Threads, 0, s>>>(a, partials, set_storage0);
    return cudaGetLastError();
}

cudaError_t launch_init64(const StepArgs64 &a, int par, const float *h, const float *v1, const float *v2,
                          cudaStream_t s)
{
    init64_kernel<<<blocks_for((long long)a.rows * a.cols), 256, 0, s>>>(a, par, h, v1, v2);
    return cudaGetLastError();
}

cudaError_t launch_extract64(const StepArgs64 &a, int par, double *h64, double *v164, double *v264, float *h32,
                             float *v132, float *v232, cudaStream_t s)
{
    extract64_kernel<<<blocks_for((long long)a.rows * a.cols), 256, 0, s>>>(a, par, h64, v164, v264, h32, v132,
                                                                          v232);
    return cudaGetLastError();
}

cudaError_t launch_extract_wide(const StepArgs &a, int par, double *h, double *v1, double *v2, cudaStream_t s)
{
    extract_wide_kernel<<<blocks_for((long long)a.rows * a.cols), 256, 0, s>>>(a, par, h, v1, v2);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const double *src, int rows, int cols, int src_pitch, float *dst, int dst_pitch,
                          cudaStream_t s)
{
    narrow_kernel<<<blocks_for((long long)rows * cols), 256, 0, s>>>(src, rows, cols, src_pitch, dst, dst_pitch);
    return cudaGetLastError();
}

cudaError_t launch_widen(const float *src, int rows, int cols, int src_pitch, double *dst, int dst_pitch,
                         cudaStream_t s)
{
    widen_kernel<<<blocks_for((long long)rows * cols), 256, 0, s>>>(src, rows, cols, src_pitch, dst, dst_pitch);
    return cudaGetLastError();
}

}  // namespace asx
