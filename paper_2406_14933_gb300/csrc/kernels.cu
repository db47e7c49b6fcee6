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

// Wave speed c = |v| + sqrt(g h) (Eq. fvm_2D_eq_frac.13) from the float32 state.
__device__ __forceinline__ float wave_speed(float v1, float v2, float h, float g)
{
    return __fadd_rn(__fsqrt_rn(__fmaf_rn(v1, v1, __fmul_rn(v2, v2))), __fsqrt_rn(__fmul_rn(g, h)));
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
    if (c->cmax_cur > 0.0f) {
        const double tau = c->cfl * c->phi / (double)c->cmax_cur;
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
    c->dtf = (float)dt;
    c->active = 1;
}

// Books the finished step (run by one thread after every CTA of the step is done).
__device__ void finish_step(DevCtl *c)
{
    volatile DevCtl *vc = c;
    const unsigned bits = vc->cmax_bits;
    const double outq = vc->out_acc;
    const double clq = vc->clamp_acc;
    const float cmax = __uint_as_float(bits);
    c->rain_in += c->sigma * (double)c->ncells * (double)c->qr;
    c->outflow += c->sigma * outq;
    c->clamped += c->sigma * clq;
    c->t = c->t_next;
    c->step += 1;
    c->parity ^= 1;
    if (c->sample_dt > 0.0 && c->t == (double)(c->n_samples + 1) * c->sample_dt) {
        if (c->n_samples < c->max_samples) c->samples[c->n_samples] = c->outflow;
        c->n_samples += 1;
    }
    if (!(cmax <= FLT_MAX)) c->err |= kErrNumeric;   // NaN or Inf somewhere
    c->cmax_cur = cmax;
    c->cmax_bits = 0u;
    c->out_acc = 0.0;
    c->clamp_acc = 0.0;
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

__device__ __forceinline__ Cell load_cell(const StepArgs &a, const float *mhi, const float *v1,
                                          const float *v2, size_t k)
{
    Cell q;
    q.m = __ldg(mhi + k);
    q.v1 = __ldg(v1 + k);
    q.v2 = __ldg(v2 + k);
    q.z = __ldg(a.z + k);
    q.h = __fdiv_rn(q.m, a.cls ? a.cls_theta[__ldg(a.cls + k)] : __ldg(a.theta + k));
    return q;
}

// Terms of the edge between A (lower index) and B, B lying in owned direction D of A
// (0 = E, 1 = NE, 2 = NW): mass increment q = kappa * l * (theta h)_(A,B) * v_n, the
// momentum flux F (v_a)_(A,B) and the pressure term P_a = -1/2 l g dw (theta h)^ n_a.
// A receives -q and -F v + P, B receives +q and +F v + P.
template <int D>
__device__ __forceinline__ void edge_terms(const Cell &A, const Cell &B, float l, float kappa,
                                           float c1, float c2, float &q, float &fa1, float &fa2,
                                           float &p1, float &p2)
{
    const float s1 = __fadd_rn(A.v1, B.v1);          // 2 (v_1)_(A,B)
    const float s2 = __fadd_rn(A.v2, B.v2);
    float vn;                                        // (v_n)_(A,B), Eq. fvm_2D_eq.04
    if (D == 0) vn = __fmul_rn(0.5f, s1);
    else if (D == 1) vn = __fmul_rn(0.5f, __fmaf_rn(kS32, s2, __fmul_rn(0.5f, s1)));
    else vn = __fmul_rn(0.5f, __fmaf_rn(kS32, s2, __fmul_rn(-0.5f, s1)));
    const float mu = vn > 0.0f ? A.m : B.m;          // Eq. fvm_2D_eq.06 (F = 0 if v_n = 0)
    const float F = __fmul_rn(__fmul_rn(l, mu), vn);
    q = __fmul_rn(kappa, F);
    const float hF = __fmul_rn(0.5f, F);
    fa1 = __fmul_rn(hF, s1);
    fa2 = __fmul_rn(hF, s2);
    const float dw = __fadd_rn(__fsub_rn(B.z, A.z), __fsub_rn(B.h, A.h));   // (w_B - w_A) / g
    const float hat = vn != 0.0f ? mu : (dw < 0.0f ? A.m : B.m);          // Eq. fvm_2D_eq.05
    const float dh = __fmul_rn(dw, hat);
    p1 = __fmul_rn(c1, dh);
    p2 = __fmul_rn(c2, dh);
}

__device__ __forceinline__ bool side_is_free(const StepArgs &a, int side, int pos)
{
    if (a.bc[side] != ASX_BC_FREE) return false;
    if (a.fb[side] == a.fe[side]) return true;
    return pos >= a.fb[side] && pos < a.fe[side];
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

// Block reduction of (max c, sum outflow, sum clamp) and the last-CTA step finish.
template <int NT>
__device__ __forceinline__ void reduce_and_finish(const StepArgs &a, float c, double outq,
                                                  double clq)
{
    __shared__ unsigned s_max[NT / 32];
    __shared__ double s_out[NT / 32], s_cl[NT / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    unsigned bits = __float_as_uint(__fadd_rn(c, 0.0f));   // -0 -> +0; NaN keeps high bits
    bits = __reduce_max_sync(0xffffffffu, bits);
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
        if (so != 0.0) atomicAdd(&ctl->out_acc, so);
        if (sc != 0.0) atomicAdd(&ctl->clamp_acc, sc);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->done_ctas, 1u);
        s_last = (prev == (unsigned)a.nblocks - 1u);
        if (s_last) {
            __threadfence();
            finish_step(ctl);
        }
    }
}

// ------------------------------------------------------------ step: gather variant

constexpr int kGX = 32, kGY = 8;

// One thread per cell: loads the cell and its six neighbours, evaluates the six edges
// (each in the canonical orientation, so a shared edge gives both cells the same
// increment), updates the cell and writes the other state buffer.
__global__ void __launch_bounds__(kGX *kGY) step_gather_kernel(const StepArgs a)
{
    const DevCtl *ctl = a.ctl;
    if (!ctl->active) return;
    const int par = ctl->parity;
    const float kappa = ctl->kappa, qr = ctl->qr, dtf = ctl->dtf;
    const float *mhi = a.mhi[par], *mlo = a.mlo[par], *v1 = a.v1[par], *v2 = a.v2[par];
    const int c = blockIdx.x * kGX + threadIdx.x;
    const int r = blockIdx.y * kGY + threadIdx.y;
    float cw = 0.0f;
    double outq = 0.0, clq = 0.0;
    if (r < a.rows && c < a.cols) {
        const size_t k = (size_t)r * a.pitch + c;
        const Cell I = load_cell(a, mhi, v1, v2, k);
        float shi = I.m, slo = __ldg(mlo + k);
        float M1 = 0.0f, M2 = 0.0f;      // J_a + S_a
        double outd = 0.0;               // booked exactly as applied (each q is a float)
#pragma unroll
        for (int d = 0; d < 6; d++) {
            int rr, cc, side;
            if (neighbour(a.rows, a.cols, r, c, d, rr, cc, side)) {
                const Cell J = load_cell(a, mhi, v1, v2, (size_t)rr * a.pitch + cc);
                float q, f1, f2, p1, p2;
                switch (d) {
                case 0: edge_terms<0>(I, J, a.l, kappa, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
                case 1: edge_terms<1>(I, J, a.l, kappa, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
                case 2: edge_terms<2>(I, J, a.l, kappa, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
                case 3: edge_terms<0>(J, I, a.l, kappa, a.cpe[0][0], a.cpe[0][1], q, f1, f2, p1, p2); break;
                case 4: edge_terms<1>(J, I, a.l, kappa, a.cpe[1][0], a.cpe[1][1], q, f1, f2, p1, p2); break;
                default: edge_terms<2>(J, I, a.l, kappa, a.cpe[2][0], a.cpe[2][1], q, f1, f2, p1, p2); break;
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
            } else {
                const int pos = (side == ASX_SIDE_S || side == ASX_SIDE_N) ? c : r;
                if (side_is_free(a, side, pos)) {
                    // free discharge: ghost copy of the cell, outflow only
                    const float vn = __fmaf_rn(I.v1, kN1[d], __fmul_rn(I.v2, kN2[d]));
                    if (vn > 0.0f) {
                        const float F = __fmul_rn(__fmul_rn(a.l, I.m), vn);
                        const float q = __fmul_rn(kappa, F);
                        acc_add(shi, slo, -q);
                        M1 -= F * I.v1;
                        M2 -= F * I.v2;
                        outd += (double)q;
                    }
                }
                // wall: mirror ghost, the edge carries nothing
            }
        }
        outq = outd;
        // rain at t^{n+1}
        acc_add(shi, slo, qr);
        float hi, lo;
        two_sum(shi, slo, hi, lo);
        if (hi < 0.0f || (hi == 0.0f && lo < 0.0f)) {
            clq = -((double)hi + (double)lo);
            hi = 0.0f;
            lo = 0.0f;
        }
        // momentum: gamma = theta h v + dt / sigma (J + S)
        const float g1 = __fmaf_rn(kappa, M1, I.m * I.v1);
        const float g2 = __fmaf_rn(kappa, M2, I.m * I.v2);
        // implicit friction: v = 2 gamma / (alpha + sqrt(alpha^2 + 4 beta |gamma|))
        float th, ka, kb;
        if (a.cls) {
            const int cl = a.cls[k];
            th = a.cls_theta[cl];
            ka = a.cls_a[cl];
            kb = a.cls_b[cl];
        } else {
            th = a.theta[k];
            ka = a.alpha_p * (1.0f - th);
            kb = th * a.alpha_s;
        }
        const float hn = __fdiv_rn(hi, th);
        const float beta = dtf * __fmaf_rn(ka, hn, kb);
        const float ng = hypotf(g1, g2);
        const float den = hi + __fsqrt_rn(__fmaf_rn(hi, hi, 4.0f * beta * ng));
        float w1 = 0.0f, w2 = 0.0f;
        if (den > 0.0f) {
            w1 = __fdiv_rn(2.0f * g1, den);
            w2 = __fdiv_rn(2.0f * g2, den);
        }
        const int np = par ^ 1;
        a.mhi[np][k] = hi;
        a.mlo[np][k] = lo;
        a.v1[np][k] = w1;
        a.v2[np][k] = w2;
        cw = wave_speed(w1, w2, hn, a.g);
    }
    reduce_and_finish<kGX * kGY>(a, cw, outq, clq);
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
    float cm = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / a.cols), c = (int)(i - (long long)r * a.cols);
        const size_t k = (size_t)r * a.pitch + c;
        const float hi = mhi[k];
        s += (double)hi + (double)mlo[k];
        const float h = __fdiv_rn(hi, cell_theta(a, k));
        cm = fmaxf(cm, wave_speed(v1[k], v2[k], h, a.g));
    }
    __shared__ double ss[kScanThreads / 32];
    __shared__ unsigned sm[kScanThreads / 32];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(__fadd_rn(cm, 0.0f)));
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
            double tot = 0.0, cmx = 0.0;
            for (unsigned b = 0; b < gridDim.x; b++) {
                tot += vp[2 * b];
                cmx = fmax(cmx, vp[2 * b + 1]);
            }
            ctl->storage = tot * ctl->sigma;
            if (set_storage0) ctl->storage0 = ctl->storage;
            ctl->cmax_cur = (float)cmx;
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
