// ensemble.cu -- batched ensembles of uneven rasters in one persistent kernel, its
// autotuner, and the asx_ensemble_* C ABI.
//
// Each scenario is an independent raster with its own time step, clock, ledger and
// hydrograph (the same step as a single raster: Sec. 2.2, Eq. fvm_2D_eq_frac.07 in the form
// of Appendix A, with the CFL step of Eqs. fvm_2D_eq_frac.12-13).  The sensitivity and
// calibration sweeps of Secs. 4.3-4.4 are ensembles of this kind.
//
// Kernel: a persistent grid of thread-block clusters.  A cluster takes the next scenario
// from an atomic queue (scenarios sorted longest first) and runs it to its end time: per
// step, the cluster's CTAs split the raster's rows, each updates its band with the gather
// cell code, reduces max wave speed / outflow / clamped water, and after one hardware
// cluster barrier every CTA reads all partials through distributed shared memory and
// derives the same next time step.  No grid-wide synchronisation and no spin wait.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

// the ensemble kernels run many steps per launch: state loads must be coherent
#define ASX_STATE_COHERENT_LOADS
#include "strip_tile.cuh"

namespace cg = cooperative_groups;

namespace asx {

constexpr int kEnsMaxRain = 8;
constexpr int kEnsMaxCluster = 8;

// Device table entry of one scenario: inputs (args, clock parameters) and results.
struct EnsScenario {
    StepArgs a;                       // geometry, state pointers, coefficients (a.ctl unused)
    double t_end, cfl, dt_max, sigma, phi, sample_dt;
    int n_rain, max_samples;
    double rain_t[kEnsMaxRain], rain_r[kEnsMaxRain];
    double *samples;                  // cumulative outflow at sample times
    // results
    double t, rain_in, outflow, clamped, storage0, storage;
    long long steps, max_steps;
    int n_samples, err, parity, pad;
};

struct EnsPartial {
    unsigned cbits;
    unsigned err;        // error bits (kErrTimeout) of the CTA's step
    double out, cl, sto;
};

namespace {

__device__ double ens_rain(const EnsScenario &s, double t)
{
    const int n = s.n_rain;
    if (n <= 0) return 0.0;
    if (t < s.rain_t[0] || t > s.rain_t[n - 1]) return 0.0;
    if (n == 1) return s.rain_r[0];
    for (int k = 0; k + 1 < n; k++) {
        const double t0 = s.rain_t[k], t1 = s.rain_t[k + 1];
        if (t <= t1) {
            if (t1 == t0) return s.rain_r[k + 1];
            return s.rain_r[k] + (s.rain_r[k + 1] - s.rain_r[k]) * (t - t0) / (t1 - t0);
        }
    }
    return s.rain_r[n - 1];
}

// Clock of the scenario a CTA is running (identical in every CTA of the cluster).
struct EnsClock {
    double t, dt, t_next, rain_in, outflow, clamped, storage0, storage;
    long long steps;
    float cmax, kappa, qr, dtf;
    int n_samples, parity, active, err;
};

// Next time step, as prepare_step does for a single raster.
__device__ void ens_prepare(const EnsScenario &s, EnsClock &k)
{
    k.active = 0;
    if (k.err) return;
    if (!(k.t < s.t_end) || k.steps >= s.max_steps) return;
    double dt = s.dt_max;
    if (k.cmax > 0.0f) {
        const double tau = s.cfl * s.phi / (double)k.cmax;
        if (tau < dt) dt = tau;
    }
    double t_stop = s.t_end;
    if (s.sample_dt > 0.0) {
        const double ns = (double)(k.n_samples + 1) * s.sample_dt;
        if (ns < t_stop) t_stop = ns;
    }
    double tn;
    if (k.t + dt >= t_stop) {
        dt = t_stop - k.t;
        tn = t_stop;
    } else {
        tn = k.t + dt;
    }
    if (!(dt > 0.0)) {           // a zero or non-finite step cannot advance the clock
        k.err |= kErrNumeric;
        return;
    }
    k.dt = dt;
    k.t_next = tn;
    k.kappa = (float)(dt / s.sigma);
    k.qr = (float)(dt * ens_rain(s, tn));
    k.dtf = (float)dt;
    k.active = 1;
}

template <int NT>
__device__ __forceinline__ void block_reduce(unsigned &cb, double &out, double &cl, double &sto)
{
    __shared__ unsigned rb[NT / 32];
    __shared__ double ro[NT / 32], rc[NT / 32], rs[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    cb = __reduce_max_sync(0xffffffffu, cb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        out += __shfl_down_sync(0xffffffffu, out, o);
        cl += __shfl_down_sync(0xffffffffu, cl, o);
        sto += __shfl_down_sync(0xffffffffu, sto, o);
    }
    __syncthreads();
    if (lane == 0) {
        rb[wid] = cb;
        ro[wid] = out;
        rc[wid] = cl;
        rs[wid] = sto;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; w++) {
            cb = max(cb, rb[w]);
            out += ro[w];
            cl += rc[w];
            sto += rs[w];
        }
    }
}

// The CTAs that run a scenario together: the whole cluster, or (solo) this CTA alone, which
// then never touches a cluster barrier or another CTA's shared memory.
struct Group {
    cg::cluster_group cluster;
    unsigned rank, size;
    bool solo;
    __device__ __forceinline__ void sync()
    {
        if (solo) __syncthreads();
        else cluster.sync();
    }
    template <class T>
    __device__ __forceinline__ T *peer(T *p, unsigned q)
    {
        return solo ? p : cluster.map_shared_rank(p, q);
    }
};

// Shared-memory state of a CTA of either ensemble kernel.
struct EnsShared {
    EnsScenario P;       // the running scenario's parameter image (P.a: its step arguments),
                         // read from here by the step's serial part instead of global memory
    EnsClock clk;        // its clock (every CTA of the cluster computes the same)
    EnsPartial part[2];  // this CTA's step partials, slots alternating by step parity
    int s_idx;           // scenario popped by the cluster's rank 0
};

// The cluster's next scenario from the queue (-1 when none is left).
__device__ __forceinline__ int ens_pop(Group &grp, EnsShared &sh, const int *order, int n_scen, unsigned *queue)
{
    if (grp.rank == 0 && threadIdx.x == 0) {
        const unsigned q = atomicAdd(queue, 1u);
        sh.s_idx = q < (unsigned)n_scen ? order[q] : -1;
    }
    grp.sync();
    const int si = *grp.peer(&sh.s_idx, 0);
    grp.sync();                  // every rank has read s_idx before rank 0 pops again
    return si;
}

// Takes scenario S: arguments and a zero clock into shared memory, then the initial scan
// (c_max and storage of the initial state over this CTA's row band [rb0, rb1)), the
// cluster-wide reduction and the first time step.
template <int NT>
__device__ void ens_start(Group &grp, EnsShared &sh, int rb0, int rb1)
{
    const unsigned csize = grp.size;
    const int tid = threadIdx.x;
    const EnsScenario &S = sh.P;
    const StepArgs &sa = sh.P.a;
    EnsClock &clk = sh.clk;
    const int cols = sa.cols, band = (rb1 - rb0) * cols;
    unsigned cb = 0u;
    double out = 0.0, cl = 0.0, sto = 0.0;
    for (int i = tid; i < band; i += NT) {
        const int r = rb0 + i / cols, c = i % cols;
        const size_t k = (size_t)r * sa.pitch + c;
        const float hi = sa.mhi[0][k];
        sto += (double)hi + (double)sa.mlo[0][k];
        const float h = __fmul_rn(hi, cell_rtheta(sa, k));
        cb = max(cb, speed_bits(wave_speed(sa.v1[0][k], sa.v2[0][k], h, sa.g)));
    }
    block_reduce<NT>(cb, out, cl, sto);
    if (tid == 0) sh.part[0] = EnsPartial{cb, 0u, 0.0, 0.0, sto};
    grp.sync();
    if (tid == 0) {
        unsigned cm = 0u;
        double st = 0.0;
        for (unsigned q = 0; q < csize; q++) {
            const EnsPartial p = *grp.peer(&sh.part[0], q);
            cm = max(cm, p.cbits);
            st += p.sto;
        }
        clk.cmax = __uint_as_float(cm);
        if (!(clk.cmax <= FLT_MAX)) clk.err |= kErrNumeric;
        clk.storage0 = st * S.sigma;
        ens_prepare(S, clk);
    }
    grp.sync();                  // part[0] is read by every rank before it is reused
}

// Ends a step: block and cluster reductions of the new wave speed (bits cb), the
// boundary and clamp sums and the error bits (err; *ctl_err is read after the block
// barrier), then the clock, ledger, hydrograph sample and next time step.
template <int NT>
__device__ void ens_step_end(Group &grp, EnsShared &sh, unsigned cb, double out, double cl, unsigned err,
                             const int *ctl_err)
{
    const unsigned rank = grp.rank, csize = grp.size;
    const int tid = threadIdx.x;
    const EnsScenario &S = sh.P;
    EnsClock &clk = sh.clk;
    const int par = clk.parity;
    double sto = 0.0;
    const int any_err = __syncthreads_or(err != 0u);
    block_reduce<NT>(cb, out, cl, sto);
    if (tid == 0) {
        unsigned eb = any_err ? (unsigned)kErrTimeout : 0u;
        if (ctl_err) eb |= (unsigned)*ctl_err;
        __threadfence();
        sh.part[par] = EnsPartial{cb, eb, out, cl, 0.0};
    }
    grp.sync();                  // the band is written and the partials are in place
    if (tid == 0) {
        unsigned cm = 0u, eb = 0u;
        double o = 0.0, c = 0.0;
        for (unsigned q = 0; q < csize; q++) {
            const EnsPartial p = *grp.peer(&sh.part[par], q);
            cm = max(cm, p.cbits);
            eb |= p.err;
            o += p.out;
            c += p.cl;
        }
        const StepArgs &sa = S.a;
        clk.rain_in += S.sigma * (double)((long long)sa.rows * sa.cols) * (double)clk.qr;
        clk.outflow += S.sigma * o;
        clk.clamped += S.sigma * c;
        clk.t = clk.t_next;
        clk.steps += 1;
        clk.parity ^= 1;
        if (S.sample_dt > 0.0 && clk.t == (double)(clk.n_samples + 1) * S.sample_dt) {
            if (rank == 0 && clk.n_samples < S.max_samples) S.samples[clk.n_samples] = clk.outflow;
            clk.n_samples += 1;
        }
        clk.cmax = __uint_as_float(cm);
        if (!(clk.cmax <= FLT_MAX)) clk.err |= kErrNumeric;
        clk.err |= (int)eb;
        ens_prepare(S, clk);
    }
    __syncthreads();
}

// Final storage of the scenario over this CTA's row band and the results (rank 0).
template <int NT>
__device__ void ens_finish(Group &grp, EnsShared &sh, EnsScenario &S, int rb0, int rb1)
{
    const unsigned rank = grp.rank, csize = grp.size;
    const int tid = threadIdx.x;
    const StepArgs &sa = sh.P.a;
    const EnsClock &clk = sh.clk;
    const int par = clk.parity, cols = sa.cols, band = (rb1 - rb0) * cols;
    unsigned cb = 0u;
    double out = 0.0, cl = 0.0, sto = 0.0;
    for (int i = tid; i < band; i += NT) {
        const int r = rb0 + i / cols, c = i % cols;
        const size_t k = (size_t)r * sa.pitch + c;
        sto += (double)sa.mhi[par][k] + (double)sa.mlo[par][k];
    }
    block_reduce<NT>(cb, out, cl, sto);
    if (tid == 0) sh.part[0] = EnsPartial{0u, 0u, 0.0, 0.0, sto};
    grp.sync();
    if (rank == 0 && tid == 0) {
        double st = 0.0;
        for (unsigned q = 0; q < csize; q++) st += grp.peer(&sh.part[0], q)->sto;
        S.t = clk.t;
        S.steps = clk.steps;
        S.rain_in = clk.rain_in;
        S.outflow = clk.outflow;
        S.clamped = clk.clamped;
        S.storage0 = clk.storage0;
        S.storage = st * S.sigma;
        S.n_samples = clk.n_samples;
        S.err = clk.err;
        S.parity = clk.parity;
    }
    grp.sync();
}

// Zero clock of a newly taken scenario (one thread).
__device__ __forceinline__ void ens_clock_zero(EnsClock &clk)
{
    clk.t = 0.0;
    clk.steps = 0;
    clk.rain_in = clk.outflow = clk.clamped = 0.0;
    clk.n_samples = 0;
    clk.parity = 0;
    clk.err = 0;
}

// The persistent gather ensemble kernel.  NT threads per CTA, K cells per thread per
// round; MODE 0: the plain scheme; 1: inflow sides (given mass flux, Dirichlet) compiled
// in; 2: inflow sides and the optional terms (artificial viscosity, linear resistance, dry
// threshold) compiled in.
// (at most 64 registers, so that 1,024 threads, e.g. two CTAs of 512, share an SM)
template <int NT, int K, int MODE>
__global__ void __launch_bounds__(NT, 1024 / NT) ensemble_kernel(EnsScenario *scen, const int *order, int n_scen,
                                                                 unsigned *queue)
{
    cg::cluster_group cluster = cg::this_cluster();
    Group grp{cluster, cluster.block_rank(), cluster.num_blocks(), false};
    const unsigned rank = grp.rank, csize = grp.size;
    __shared__ EnsShared sh;
    const StepArgs &sa = sh.P.a;
    EnsClock &clk = sh.clk;
    const int tid = threadIdx.x;
    for (;;) {
        const int si = ens_pop(grp, sh, order, n_scen, queue);
        if (si < 0) return;
        EnsScenario &S = scen[si];
        if (tid == 0) {
            sh.P = S;
            ens_clock_zero(clk);
        }
        __syncthreads();
        const int rows = sa.rows, cols = sa.cols;
        const int rb0 = (int)(((long long)rows * rank) / csize);
        const int rb1 = (int)(((long long)rows * (rank + 1)) / csize);
        const int band = (rb1 - rb0) * cols;
        ens_start<NT>(grp, sh, rb0, rb1);
        __syncthreads();
        // ---- time loop
        while (clk.active) {
            StepScalars sc;
            sc.par = clk.parity;
            sc.kappa = clk.kappa;
            sc.qr = clk.qr;
            sc.dtf = clk.dtf;
            sc.kl2 = sc.kappa * (0.5f * sa.l);
            sc.l4 = 0.25f * sa.l;
            sc.l2 = 0.5f * sa.l;
            unsigned cb = 0u;
            FF outd, clq;
            for (int i0 = tid; i0 < band; i0 += NT * K) {
#pragma unroll
                for (int u = 0; u < K; u++) {
                    const int i = i0 + u * NT;
                    if (i < band)
                        gather_cell<(MODE >= 2), (MODE >= 1)>(sa, sc, rb0 + i / cols, i % cols, cb, outd, clq);
                }
            }
            ens_step_end<NT>(grp, sh, cb, outd.value(), clq.value(), 0u, nullptr);
        }
        ens_finish<NT>(grp, sh, S, rb0, rb1);
    }
}

// The persistent strip ensemble kernel: NW warps per CTA, each a strip tile worker with
// its own TMA ring (strip_tile.cuh).  Per step the scenario's units (tiles of 128 columns
// x tile_rows rows, then the frame in blocks of kFrameCells cells: the units the single
// raster's strip kernel gives its CTAs) are dealt to the group's CTAs by index modulo the
// group size, and within a CTA each warp takes the next one when it is free; every cell
// is computed by the same code, hence to the same bits, as in a single raster with the
// same tile height.  The tile code reads the step's scalars and reports copy errors
// through a control block in shared memory; tensor maps per scenario live in global
// memory.  Each thread fences its stores to the async proxy before the barrier that ends
// the step, so the next step's tensor loads see them.
// Two phases: the first n_big scenarios of `order` run on whole clusters (popped from
// queue[0]); once they are all taken, every CTA of the cluster runs the remaining
// scenarios alone (popped from queue[1]), with CTA barriers only.
template <int NW, bool EXT>
__global__ void __launch_bounds__(NW * 32, NW <= 16 ? 16 / NW : 1) ensemble_strip_kernel(EnsScenario *scen, const StripMaps *maps,
                                                                          const int *order, int n_scen, int n_big,
                                                                          unsigned *queue)
{
    constexpr int NT = NW * 32;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    StripSmem<false> *rings =
        reinterpret_cast<StripSmem<false> *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ EnsShared sh;
    __shared__ DevCtl sctl;                          // step scalars and error word of the tile code
    __shared__ int s_cur;                            // index of the running scenario
    __shared__ float s_cls[3][kMaxClasses];          // class tables (unused: per-cell theta)
    __shared__ int s_next;                           // next unit of this CTA in the running step
    __shared__ unsigned s_grank, s_gsize;            // this CTA's rank and size of its group
    __shared__ int s_solo;                           // the group is this CTA alone
    // the group, rebuilt from shared memory where it is needed (not held in registers
    // through the tile code)
    auto group = [&]() { return Group{cluster, s_grank, s_gsize, s_solo != 0}; };
    StepArgs &sa = sh.P.a;
    EnsClock &clk = sh.clk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    StripSmem<false> &R = rings[warp];
    bool ring_used = false;              // this warp's ring barriers hold a previous tile's phases
    for (int phase = 0; phase < 2; phase++) {
        if (tid == 0) {
            s_solo = phase;
            s_grank = phase ? 0u : cluster.block_rank();
            s_gsize = phase ? 1u : cluster.num_blocks();
        }
        __syncthreads();
        for (;;) {
            {
                Group grp = group();
                const int si = phase == 0 ? ens_pop(grp, sh, order, n_big, queue)
                                          : ens_pop(grp, sh, order + n_big, n_scen - n_big, queue + 1);
                if (si < 0) break;
                if (tid == 0) {
                    sh.P = scen[si];
                    sa.ctl = &sctl;
                    sctl.err = 0;
                    s_cur = si;
                    ens_clock_zero(clk);
                }
                __syncthreads();
                // the initial scan over this CTA's row band
                ens_start<NT>(grp, sh, (int)(((long long)sa.rows * grp.rank) / grp.size),
                              (int)(((long long)sa.rows * (grp.rank + 1)) / grp.size));
                __syncthreads();
            }
            // the scenario index lives in shared memory, not in registers, through the time loop
            const StripMaps &M = maps[s_cur];
            const int ns = sa.nstrips + (sa.cx_last >= 0 ? 1 : 0);
            if (lane == 0 && sa.ntiles > 0) {
                // the scenario's maps, written to global memory by the host, for this warp's
                // tensor copies
                for (int p = 0; p < 2; p++) {
                    tensormap_acquire(&M.mhi[p]);
                    tensormap_acquire(&M.v1[p]);
                    tensormap_acquire(&M.v2[p]);
                    tensormap_acquire(&M.mlo[p]);
                }
                tensormap_acquire(&M.z);
                tensormap_acquire(&M.th);
            }
            // ---- time loop
            while (clk.active) {
                if (tid == 0) {
                    sctl.parity = clk.parity;
                    sctl.kappa = clk.kappa;
                    sctl.qr = clk.qr;
                    sctl.dtf = clk.dtf;
                    s_next = 0;
                }
                __syncthreads();
                // one worker per warp and step, moved from tile to tile; its reductions
                // collect the frame units' too
                Tile<false, EXT> T(sa, R, s_cls, M, sa.cx0, sa.ry0, sa.cx0, sa.ry0);
                unsigned err = 0u;
                // this CTA's units are rank, rank + size, ...: its warps take them in order
                // (the tiles, then the cheaper frame blocks) as they become free
                for (;;) {
                    int j = 0;
                    if (lane == 0) j = atomicAdd(&s_next, 1);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    const int u = (int)s_grank + j * (int)s_gsize;
                    if (u >= sa.nblocks) break;
                    if (u < sa.ntiles) {
                        const int strip = u % ns, rblk = u / ns;
                        const int c0 = strip < sa.nstrips ? sa.cx0 + strip * kSW : sa.cx_last;
                        const int own_c = strip < sa.nstrips ? c0 : sa.cx0 + sa.nstrips * kSW;
                        const int r0 = rblk < sa.nrb ? sa.ry0 + rblk * sa.tile_rows : sa.r_last;
                        const int own_r = rblk < sa.nrb ? r0 : sa.ry0 + sa.nrb * sa.tile_rows;
                        if ((r0 & 1) == 0) {     // the layout puts every tile on an odd first row
                            err = kErrTimeout;
                            break;
                        }
                        // the previous tile's ring reads are done before new copies land in it,
                        // and its barriers (every copy waited for) are reset for the new tile
                        __syncwarp();
                        if (ring_used && lane == 0)
                            for (int k = 0; k < kNC; k++) mbar_inval(&R.bar[k]);
                        ring_used = true;
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        T.place(c0, r0, own_c, own_r);
                        T.run();
                        if (__any_sync(0xffffffffu, T.timed_out)) {
                            // a tensor copy did not arrive in time: wait (bounded) for the
                            // copies still in flight and stop the scenario with an error
                            if (lane == 0)
                                for (int k = max(0, T.n_issued - kNC); k < T.n_issued; k++)
                                    mbar_wait_bounded(&R.bar[k % kNC], (unsigned)((k / kNC) & 1));
                            err = kErrTimeout;
                            break;
                        }
                    } else {
                        frame_cells<EXT>(sa, (long long)(u - sa.ntiles) * kFrameCells, T.cwb, T.outd, T.clq);
                    }
                }
                const unsigned cb = T.cwb;
                const double out = T.outd.value(), cl = T.clq.value();
                asm volatile("fence.proxy.async.global;" ::: "memory");
                Group grp = group();
                ens_step_end<NT>(grp, sh, cb, out, cl, err, &sctl.err);
            }
            Group grp = group();
            ens_finish<NT>(grp, sh, scen[s_cur], (int)(((long long)sa.rows * grp.rank) / grp.size),
                           (int)(((long long)sa.rows * (grp.rank + 1)) / grp.size));
        }
    }
}

using EnsKernel = void (*)(EnsScenario *, const int *, int, unsigned *);
using EnsStripKernel = void (*)(EnsScenario *, const StripMaps *, const int *, int, int, unsigned *);

template <int NT, int K, int MODE>
EnsKernel ens_kernel_ptr()
{
    return ensemble_kernel<NT, K, MODE>;
}

template <int MODE>
EnsKernel ens_kernel_m(int nt, int k)
{
    if (nt == 256)
        return k == 1 ? ens_kernel_ptr<256, 1, MODE>() : k == 2 ? ens_kernel_ptr<256, 2, MODE>() : ens_kernel_ptr<256, 4, MODE>();
    if (nt == 512)
        return k == 1 ? ens_kernel_ptr<512, 1, MODE>() : k == 2 ? ens_kernel_ptr<512, 2, MODE>() : ens_kernel_ptr<512, 4, MODE>();
    return k == 1 ? ens_kernel_ptr<128, 1, MODE>() : k == 2 ? ens_kernel_ptr<128, 2, MODE>() : ens_kernel_ptr<128, 4, MODE>();
}

EnsKernel ens_kernel(int nt, int k, int mode)
{
    return mode >= 2 ? ens_kernel_m<2>(nt, k) : mode == 1 ? ens_kernel_m<1>(nt, k) : ens_kernel_m<0>(nt, k);
}

// Strip kernel of `threads` threads (128: 4 tile workers, 256: 8, 512: 16) with or without the
// optional terms; inflow sides are frame cells, whose gather code always has them.
EnsStripKernel ens_strip_kernel(int threads, int mode)
{
    if (mode >= 2)
        return threads == 128 ? ensemble_strip_kernel<4, true>
                              : threads == 256 ? ensemble_strip_kernel<8, true> : ensemble_strip_kernel<16, true>;
    return threads == 128 ? ensemble_strip_kernel<4, false>
                          : threads == 256 ? ensemble_strip_kernel<8, false> : ensemble_strip_kernel<16, false>;
}

size_t ens_strip_smem(int threads) { return (size_t)(threads / 32) * sizeof(StripSmem<false>) + 128; }

}  // namespace
}  // namespace asx

using namespace asx;

// ------------------------------------------------------------------ host side

struct asx_ensemble {
    int n = 0, device = 0;
    cudaStream_t stream = nullptr;
    std::vector<asx_scenario_desc> desc;
    std::vector<EnsScenario> host;          // parameter image of the device table
    std::vector<size_t> plane_off;          // float offset of each scenario's planes
    std::vector<int> pitch;
    float *buf = nullptr;
    double *samples = nullptr;
    EnsScenario *dev = nullptr;
    int *order = nullptr;
    unsigned *queue = nullptr;
    asx_ensemble_tuning tuning{};
    bool tuned = false, have_fields_all = false;
    int mode = 0;                           // kernel variant: 1 inflow sides, 2 also optional terms
    std::vector<char> have_fields;
    std::vector<long long> work_steps;      // step counts of the last complete run
    bool have_steps = false;
    StripMaps *maps = nullptr;              // per scenario: the strip kernel's tensor maps
    std::vector<char> maps_ok;              // scenario wide enough for strip tiles
    long long layout_key = -1;              // strip layout in `dev`: tile height (and shape if per scenario)
    std::vector<int> order_host;            // the queue order uploaded to `order`
    cudaGraphExec_t graph = nullptr;
    asx_ensemble_tuning graph_tuning{};
    std::string err;
};

namespace {

asx_status efail(asx_ensemble *e, asx_status st, const std::string &m)
{
    if (e) e->err = m;
    return st;
}

#define ENS_CUDA(e, call)                                                                      \
    do {                                                                                       \
        cudaError_t x_ = (call);                                                               \
        if (x_ != cudaSuccess)                                                                 \
            return efail((e), ASX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(x_));   \
    } while (0)

bool tuning_valid(const asx_ensemble_tuning &t)
{
    const bool c = t.cluster == 1 || t.cluster == 2 || t.cluster == 4 || t.cluster == kEnsMaxCluster;
    if (t.split < 0 || (t.split > 0 && (t.tile_rows == 0 || t.cluster < 2))) return false;
    if (t.tile_rows != 0) {
        const bool h = t.tile_rows == 1 || t.tile_rows == 8 || t.tile_rows == 16 || t.tile_rows == 32;
        return c && h && (t.threads == 128 || t.threads == 256 || t.threads == 512) && t.cells_per_thread == 1;
    }
    const bool n = t.threads == 128 || t.threads == 256 || t.threads == 512;
    const bool k = t.cells_per_thread == 1 || t.cells_per_thread == 2 || t.cells_per_thread == 4;
    return c && n && k;
}

// Kernel of a launch shape and its dynamic shared memory (set as the kernel's limit).
const void *shape_kernel(const asx_ensemble_tuning &t, int mode, size_t &smem)
{
    smem = 0;
    if (t.tile_rows == 0) return (const void *)ens_kernel(t.threads, t.cells_per_thread, mode);
    const void *f = (const void *)ens_strip_kernel(t.threads, mode);
    smem = ens_strip_smem(t.threads);
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return f;
}

// Clusters of this shape that fit on the device at once.
int resident_clusters(const asx_ensemble_tuning &t, int mode)
{
    size_t smem = 0;
    const void *f = shape_kernel(t, mode, smem);
    cudaLaunchConfig_t cfg{};
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = t.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(t.cluster);
    cfg.blockDim = dim3(t.threads);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, f, &cfg) != cudaSuccess || nc < 1) nc = 1;
    return nc;
}

// Strip layout of scenario i for tile height H (interior tiles and frame); scenarios too
// narrow for a tile (or without tensor maps) are all frame, taken row by row.
void scenario_layout(asx_ensemble *e, int i, int H)
{
    StepArgs &a = e->host[i].a;
    a.tile_rows = H;
    step_strip_layout(a);
    if (!e->maps_ok[i] || a.ntiles == 0) {
        const long long n = (long long)a.rows * a.cols;
        a.nstrips = a.nrb = a.ntiles = 0;
        a.cx_last = a.r_last = -1;
        a.cxe = a.cx0;
        a.rye = a.ry0;
        a.frame_n = a.frame_a = n;
        a.nblocks = (int)((n + kFrameCells - 1) / kFrameCells);
    }
}

// Modelled duration of one step of scenario i's current layout on clusters of `csize`
// CTAs of `nw` warps, in cell-updates of tile code: the units are dealt to the CTAs by
// index modulo the cluster size and, within a CTA, taken in order by the first free warp.
// A tile costs its rows with the two halo rows plus a ring start-up of ~100 cells; a
// frame cell ~3 (gather code).
double modelled_step(const asx_ensemble *e, int i, int csize, int nw)
{
    const StepArgs &a = e->host[i].a;
    const double tile = (double)(a.tile_rows + 2) * kStripW + 100.0, frame = 3.0 * kFrameCells;
    double worst = 0.0;
    std::vector<double> load((size_t)nw);
    for (int r = 0; r < csize; r++) {
        std::fill(load.begin(), load.end(), 0.0);
        for (int u = r; u < a.nblocks; u += csize) {
            auto w = std::min_element(load.begin(), load.end());
            *w += u < a.ntiles ? tile : frame;
        }
        worst = std::max(worst, *std::max_element(load.begin(), load.end()));
    }
    return worst;
}

// The scenario table's strip layout for tile height H, if it holds another: H = 8, 16 or
// 32 for every scenario, H = 1 the height of 8, 16, 32 whose modelled step is shortest on
// clusters of `csize` CTAs of `nw` warps, per scenario (H = 0, the gather kernel, needs
// none).
cudaError_t ensure_layout(asx_ensemble *e, int H, int csize, int nw, int split)
{
    const long long key = H == 1 ? 1 + 1000LL * csize + 100000LL * nw + 100000000LL * split : H;
    if (H == 0 || e->layout_key == key) return cudaSuccess;
    std::vector<int> pos(e->n);
    for (int q = 0; q < e->n; q++) pos[e->order_host[q]] = q;
    for (int i = 0; i < e->n; i++) {
        if (H != 1) {
            scenario_layout(e, i, H);
            continue;
        }
        // the group that runs scenario i: a whole cluster, or one CTA after the split
        const int gs = split > 0 && pos[i] >= split ? 1 : csize;
        int best = 32;
        double best_t = 0.0;
        for (int h : {32, 16, 8}) {
            scenario_layout(e, i, h);
            const double t = modelled_step(e, i, gs, nw);
            if (h == 32 || t < best_t) {
                best = h;
                best_t = t;
            }
        }
        scenario_layout(e, i, best);
    }
    cudaError_t x = cudaMemcpy(e->dev, e->host.data(), e->n * sizeof(EnsScenario), cudaMemcpyHostToDevice);
    e->layout_key = x == cudaSuccess ? key : -1;
    return x;
}

cudaError_t ensure_layout(asx_ensemble *e, const asx_ensemble_tuning &t)
{
    return ensure_layout(e, t.tile_rows, t.cluster, t.threads / 32, t.split);
}

cudaError_t launch_ensemble(asx_ensemble *e, const asx_ensemble_tuning &t, cudaStream_t s)
{
    size_t smem = 0;
    const void *f = shape_kernel(t, e->mode, smem);
    const int nc = std::min(resident_clusters(t, e->mode), e->n);
    cudaLaunchConfig_t cfg{};
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = t.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(nc * t.cluster);
    cfg.blockDim = dim3(t.threads);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t x = cudaMemsetAsync(e->queue, 0, 2 * sizeof(unsigned), s);
    if (x != cudaSuccess) return x;
    (void)f;
    if (t.tile_rows == 0)
        return cudaLaunchKernelEx(&cfg, ens_kernel(t.threads, t.cells_per_thread, e->mode), e->dev,
                                  (const int *)e->order, e->n, e->queue);
    const int n_big = t.split > 0 ? std::min(t.split, e->n) : e->n;
    return cudaLaunchKernelEx(&cfg, ens_strip_kernel(t.threads, e->mode), e->dev, (const StripMaps *)e->maps,
                              (const int *)e->order, e->n, n_big, e->queue);
}

// Restores every scenario's initial state and clock (the state lives in parity 0 and a
// copy of it in the spare planes at the end of the buffer).
cudaError_t reset_state(asx_ensemble *e, cudaStream_t s)
{
    for (int i = 0; i < e->n; i++) {
        EnsScenario &h = e->host[i];
        const size_t plane = (size_t)h.a.rows * e->pitch[i] * sizeof(float);
        const float *init = e->buf + e->plane_off[i] + 10 * (size_t)h.a.rows * e->pitch[i];
        for (int f = 0; f < 4; f++) {
            float *dst = f == 0 ? h.a.mhi[0] : f == 1 ? h.a.mlo[0] : f == 2 ? h.a.v1[0] : h.a.v2[0];
            cudaError_t x = cudaMemcpyAsync(dst, init + f * plane / sizeof(float), plane, cudaMemcpyDeviceToDevice, s);
            if (x != cudaSuccess) return x;
        }
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

asx_status asx_create_ensemble(int n, const asx_scenario_desc *descs, void *cuda_stream, int device,
                               asx_ensemble **out)
{
    if (!out || n < 1 || !descs) return ASX_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        const asx_scenario_desc &d = descs[i];
        if (d.rows < 2 || d.cols < 2 || (long long)d.rows * d.cols >= (1LL << 31) || !(d.edge_m > 0)) return ASX_EINVAL;
        for (int s = 0; s < 4; s++) {
            if (d.bc[s] < ASX_BC_WALL || d.bc[s] > ASX_BC_DIRICHLET) return ASX_EINVAL;
            if (!(d.bc_q[s] >= 0) || !std::isfinite(d.bc_q[s]) || !(d.bc_h[s] >= 0) || !std::isfinite(d.bc_h[s]) ||
                !std::isfinite(d.bc_u[s]))
                return ASX_EINVAL;
        }
        if (!(d.g > 0) || !(d.cfl > 0) || !(d.cfl <= 1) || !(d.dt_max > 0) || !(d.alpha_s >= 0) || !(d.alpha_p >= 0))
            return ASX_EINVAL;
        if (d.n_rain < 0 || d.n_rain > kEnsMaxRain || (d.n_rain > 0 && (!d.rain_t || !d.rain_r))) return ASX_EINVAL;
        if (!(d.t_end >= 0) || !std::isfinite(d.t_end) || !(d.sample_dt >= 0) || d.max_samples < 0) return ASX_EINVAL;
        if ((d.viscosity != 0 && d.viscosity != 1) || !(d.tau >= 0) || !std::isfinite(d.tau) || !(d.h_dry >= 0) ||
            !std::isfinite(d.h_dry))
            return ASX_EINVAL;
    }
    asx_ensemble *e = new (std::nothrow) asx_ensemble();
    if (!e) return ASX_ENOMEM;
    e->n = n;
    e->device = device;
    e->stream = (cudaStream_t)cuda_stream;
    e->desc.assign(descs, descs + n);
    for (int i = 0; i < n; i++) {
        for (int sd = 0; sd < 4; sd++)
            if (descs[i].bc[sd] == ASX_BC_FLUX || descs[i].bc[sd] == ASX_BC_DIRICHLET) e->mode = std::max(e->mode, 1);
        if (descs[i].viscosity || descs[i].tau > 0 || descs[i].h_dry > 0) e->mode = 2;
    }
    e->have_fields.assign(n, 0);
    if (cudaSetDevice(device) != cudaSuccess) { delete e; return ASX_ECUDA; }
    // planes per scenario: 8 state (2 parities x m_hi, m_lo, v1, v2), z, theta, 4 initial
    size_t total = 0, total_samples = 0;
    e->plane_off.resize(n);
    e->pitch.resize(n);
    for (int i = 0; i < n; i++) {
        e->pitch[i] = (descs[i].cols + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
        e->plane_off[i] = total;
        total += 14 * (size_t)descs[i].rows * e->pitch[i];
        total_samples += (size_t)std::max(descs[i].max_samples, 1);
    }
    cudaError_t x = cudaMalloc(&e->buf, total * sizeof(float));
    if (x == cudaSuccess) x = cudaMalloc(&e->samples, total_samples * sizeof(double));
    if (x == cudaSuccess) x = cudaMalloc(&e->dev, n * sizeof(EnsScenario));
    if (x == cudaSuccess) x = cudaMalloc(&e->order, n * sizeof(int));
    if (x == cudaSuccess) x = cudaMalloc(&e->queue, 2 * sizeof(unsigned));
    if (x == cudaSuccess) x = cudaMalloc(&e->maps, n * sizeof(StripMaps));
    if (x == cudaSuccess) x = cudaMemsetAsync(e->buf, 0, total * sizeof(float), e->stream);
    if (x != cudaSuccess) {
        asx_destroy_ensemble(e);
        return x == cudaErrorMemoryAllocation ? ASX_ENOMEM : ASX_ECUDA;
    }
    e->host.resize(n);
    size_t soff = 0;
    std::vector<int> ord(n);
    for (int i = 0; i < n; i++) {
        const asx_scenario_desc &d = descs[i];
        EnsScenario &h = e->host[i];
        std::memset(&h, 0, sizeof(h));
        StepArgs &a = h.a;
        const size_t pe = (size_t)d.rows * e->pitch[i];
        float *b = e->buf + e->plane_off[i];
        a.rows = d.rows;
        a.cols = d.cols;
        a.pitch = e->pitch[i];
        for (int p = 0; p < 2; p++) {
            a.mhi[p] = b + (4 * p + 0) * pe;
            a.mlo[p] = b + (4 * p + 1) * pe;
            a.v1[p] = b + (4 * p + 2) * pe;
            a.v2[p] = b + (4 * p + 3) * pe;
        }
        a.z = b + 8 * pe;
        a.theta = b + 9 * pe;
        a.cls = nullptr;
        a.alpha_s = (float)d.alpha_s;
        a.alpha_p = (float)d.alpha_p;
        a.l = (float)d.edge_m;
        a.g = (float)d.g;
        const double s3 = std::sqrt(3.0) / 2.0;
        const double n1[3] = {1.0, 0.5, -0.5}, n2[3] = {0.0, s3, s3};
        for (int k = 0; k < 3; k++) {
            a.cpe[k][0] = (float)(-0.5 * d.edge_m * d.g * n1[k]);
            a.cpe[k][1] = (float)(-0.5 * d.edge_m * d.g * n2[k]);
            // the strip tiles' form: momentum sums in units of l/8
            a.cpm[k][0] = (float)(-4.0 * d.g * n1[k]);
            a.cpm[k][1] = (float)(-4.0 * d.g * n2[k]);
        }
        for (int s = 0; s < 4; s++) {
            a.bc[s] = d.bc[s];
            a.fb[s] = d.free_begin[s];
            a.fe[s] = d.free_end[s];
            a.bq[s] = (float)d.bc_q[s];
            a.bhc[s] = (float)std::cbrt(d.bc_q[s] * d.bc_q[s] / d.g);
            a.bh[s] = (float)d.bc_h[s];
            a.bu[s] = (float)d.bc_u[s];
        }
        a.visc = d.viscosity;
        a.tau = (float)d.tau;
        a.h_dry = (float)d.h_dry;
        h.t_end = d.t_end;
        h.cfl = d.cfl;
        h.dt_max = d.dt_max;
        h.sigma = 1.5 * std::sqrt(3.0) * d.edge_m * d.edge_m;
        h.phi = h.sigma / (6.0 * d.edge_m);
        h.sample_dt = d.sample_dt;
        h.n_rain = d.n_rain;
        for (int k = 0; k < d.n_rain; k++) {
            h.rain_t[k] = d.rain_t[k];
            h.rain_r[k] = d.rain_r[k];
        }
        h.max_samples = d.max_samples;
        h.samples = e->samples + soff;
        soff += (size_t)std::max(d.max_samples, 1);
        h.max_steps = d.max_steps > 0 ? d.max_steps : (1LL << 62);
        ord[i] = i;
    }
    // tensor maps of the strip kernel, for the scenarios wide enough for a tile and its
    // halo columns (the others are all frame)
    std::vector<StripMaps> hmaps(n);
    e->maps_ok.assign(n, 0);
    for (int i = 0; i < n; i++) {
        const StepArgs &a = e->host[i].a;
        std::memset(&hmaps[i], 0, sizeof(StripMaps));
        if (a.cols >= kStripW + 16 && a.rows >= 4) {
            if (!make_strip_maps(hmaps[i], a, a.rows, a.cols, a.pitch)) {
                asx_destroy_ensemble(e);
                return ASX_ECUDA;
            }
            e->maps_ok[i] = 1;
        }
    }
    x = cudaMemcpyAsync(e->maps, hmaps.data(), n * sizeof(StripMaps), cudaMemcpyHostToDevice, e->stream);
    if (x != cudaSuccess) {
        asx_destroy_ensemble(e);
        return ASX_ECUDA;
    }
    // longest first: cells x expected steps ~ cells x t_end / cell size
    std::sort(ord.begin(), ord.end(), [&](int p, int q) {
        const double wp = (double)descs[p].rows * descs[p].cols * descs[p].t_end / descs[p].edge_m;
        const double wq = (double)descs[q].rows * descs[q].cols * descs[q].t_end / descs[q].edge_m;
        return wp > wq;
    });
    e->order_host = ord;
    x = cudaMemcpyAsync(e->order, ord.data(), n * sizeof(int), cudaMemcpyHostToDevice, e->stream);
    if (x == cudaSuccess)
        x = cudaMemcpyAsync(e->dev, e->host.data(), n * sizeof(EnsScenario), cudaMemcpyHostToDevice, e->stream);
    if (x == cudaSuccess) x = cudaStreamSynchronize(e->stream);
    if (x != cudaSuccess) {
        asx_destroy_ensemble(e);
        return ASX_ECUDA;
    }
    e->tuning = asx_ensemble_tuning{4, 256, 2};
    *out = e;
    return ASX_OK;
}

asx_status asx_destroy_ensemble(asx_ensemble *e)
{
    if (!e) return ASX_OK;
    cudaSetDevice(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    cudaFree(e->buf);
    cudaFree(e->samples);
    cudaFree(e->dev);
    cudaFree(e->order);
    cudaFree(e->queue);
    cudaFree(e->maps);
    delete e;
    return ASX_OK;
}

const char *asx_ensemble_last_error(const asx_ensemble *e)
{
    return e ? e->err.c_str() : "null ensemble handle";
}

asx_status asx_ensemble_set_fields(asx_ensemble *e, int s, const double *z, const float *theta,
                                   const float *h0, const float *v1, const float *v2, int kind)
{
    if (!e) return ASX_EINVAL;
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    if (!z || !theta || !h0) return efail(e, ASX_EINVAL, "z, theta and h0 are required");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return efail(e, ASX_EINVAL, "bad ptr_kind");
    const asx_scenario_desc &d = e->desc[s];
    const size_t n = (size_t)d.rows * d.cols;
    if (kind == ASX_PTR_HOST) {
        for (size_t i = 0; i < n; i++) {
            if (!std::isfinite(z[i]) || !(theta[i] > 0.0f) || !(theta[i] <= 1.0f) || !(h0[i] >= 0.0f) ||
                !std::isfinite(h0[i]) || (v1 && !std::isfinite(v1[i])) || (v2 && !std::isfinite(v2[i])))
                return efail(e, ASX_EINVAL, "field value out of range");
        }
    }
    ENS_CUDA(e, cudaSetDevice(e->device));
    const int pitch = e->pitch[s];
    const cudaMemcpyKind mk = kind == ASX_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    auto put = [&](void *dst, const void *src) {
        return cudaMemcpy2DAsync(dst, (size_t)pitch * 4, src, (size_t)d.cols * 4, (size_t)d.cols * 4, d.rows, mk,
                                 e->stream);
    };
    EnsScenario &h = e->host[s];
    StepArgs &a = h.a;
    // the bed rounded to the nearest float32
    if (kind == ASX_PTR_HOST) {
        std::vector<float> zf(n);
        for (size_t i = 0; i < n; i++) zf[i] = (float)z[i];
        ENS_CUDA(e, put((void *)a.z, zf.data()));
        ENS_CUDA(e, cudaStreamSynchronize(e->stream));      // zf is released on return
    } else {
        ENS_CUDA(e, launch_narrow(z, d.rows, d.cols, d.cols, (float *)a.z, pitch, e->stream));
    }
    ENS_CUDA(e, put((void *)a.theta, theta));
    ENS_CUDA(e, put(a.mhi[1], h0));
    if (v1) ENS_CUDA(e, put(a.v1[1], v1));
    else ENS_CUDA(e, cudaMemsetAsync(a.v1[1], 0, (size_t)d.rows * pitch * 4, e->stream));
    if (v2) ENS_CUDA(e, put(a.v2[1], v2));
    else ENS_CUDA(e, cudaMemsetAsync(a.v2[1], 0, (size_t)d.rows * pitch * 4, e->stream));
    ENS_CUDA(e, launch_init_state(a, 0, a.mhi[1], a.v1[1], a.v2[1], e->stream));
    // keep a copy of the initial state for repeated runs
    const size_t plane = (size_t)d.rows * pitch;
    float *init = e->buf + e->plane_off[s] + 10 * plane;
    ENS_CUDA(e, cudaMemcpyAsync(init, a.mhi[0], plane * 4, cudaMemcpyDeviceToDevice, e->stream));
    ENS_CUDA(e, cudaMemcpyAsync(init + plane, a.mlo[0], plane * 4, cudaMemcpyDeviceToDevice, e->stream));
    ENS_CUDA(e, cudaMemcpyAsync(init + 2 * plane, a.v1[0], plane * 4, cudaMemcpyDeviceToDevice, e->stream));
    ENS_CUDA(e, cudaMemcpyAsync(init + 3 * plane, a.v2[0], plane * 4, cudaMemcpyDeviceToDevice, e->stream));
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    e->have_fields[s] = 1;
    e->have_fields_all = std::all_of(e->have_fields.begin(), e->have_fields.end(), [](char c) { return c != 0; });
    return ASX_OK;
}

asx_status asx_ensemble_run(asx_ensemble *e, const asx_ensemble_tuning *tuning)
{
    if (!e) return ASX_EINVAL;
    if (!e->have_fields_all) return efail(e, ASX_ESTATE, "asx_ensemble_set_fields missing for a scenario");
    const asx_ensemble_tuning t = tuning ? *tuning : e->tuning;
    if (!tuning_valid(t)) return efail(e, ASX_EINVAL, "tuning out of range");
    ENS_CUDA(e, cudaSetDevice(e->device));
    ENS_CUDA(e, reset_state(e, e->stream));
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    ENS_CUDA(e, ensure_layout(e, t));
    // one persistent launch, captured once per tuning in a CUDA graph and replayed
    if (!e->graph || std::memcmp(&e->graph_tuning, &t, sizeof(t)) != 0) {
        if (e->graph) {
            cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
        }
        cudaStream_t cs;
        ENS_CUDA(e, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t x = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (x == cudaSuccess) {
            x = launch_ensemble(e, t, cs);
            cudaError_t x2 = cudaStreamEndCapture(cs, &g);
            if (x == cudaSuccess) x = x2;
        }
        if (x == cudaSuccess) x = cudaGraphInstantiate(&e->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (x != cudaSuccess) {
            e->graph = nullptr;
            return efail(e, ASX_ECUDA, std::string("ensemble graph: ") + cudaGetErrorString(x));
        }
        e->graph_tuning = t;
    }
    ENS_CUDA(e, cudaGraphLaunch(e->graph, e->stream));
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    // read back the results
    std::vector<EnsScenario> res(e->n);
    ENS_CUDA(e, cudaMemcpy(res.data(), e->dev, e->n * sizeof(EnsScenario), cudaMemcpyDeviceToHost));
    bool bad = false, timed_out = false;
    for (int i = 0; i < e->n; i++) {
        EnsScenario &h = e->host[i];
        h.t = res[i].t;
        h.steps = res[i].steps;
        h.rain_in = res[i].rain_in;
        h.outflow = res[i].outflow;
        h.clamped = res[i].clamped;
        h.storage0 = res[i].storage0;
        h.storage = res[i].storage;
        h.n_samples = res[i].n_samples;
        h.err = res[i].err;
        h.parity = res[i].parity;
        if (h.err & kErrTimeout) timed_out = true;
        else if (h.err) bad = true;
    }
    if (timed_out) return efail(e, ASX_ETIMEOUT, "a tensor copy of the strip kernel did not arrive in time");
    if (bad) return efail(e, ASX_ENUMERIC, "a scenario's state became non-finite");
    // A run that took every scenario to its end time gives the real work of each (cells x
    // steps; the step sequence does not depend on the launch shape).  Later runs take the
    // scenarios longest first by that work, and the autotuner cuts them in its proportion.
    bool complete = true;
    for (int i = 0; i < e->n; i++)
        if (!(e->host[i].t >= e->host[i].t_end)) complete = false;
    if (complete) {
        e->work_steps.resize(e->n);
        for (int i = 0; i < e->n; i++) e->work_steps[i] = e->host[i].steps;
        e->have_steps = true;
        std::vector<int> ord(e->n);
        for (int i = 0; i < e->n; i++) ord[i] = i;
        auto work = [&](int i) { return (double)e->desc[i].rows * e->desc[i].cols * (double)e->work_steps[i]; };
        std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) { return work(p) > work(q); });
        ENS_CUDA(e, cudaMemcpy(e->order, ord.data(), e->n * sizeof(int), cudaMemcpyHostToDevice));
        if (ord != e->order_host) e->layout_key = -1;   // per-scenario layouts follow the order
        e->order_host = ord;
    }
    return ASX_OK;
}

asx_status asx_ensemble_autotune(asx_ensemble *e, int max_steps, asx_ensemble_tuning *best_out)
{
    if (!e || max_steps < 1) return ASX_EINVAL;
    if (!e->have_fields_all) return efail(e, ASX_ESTATE, "asx_ensemble_set_fields missing for a scenario");
    ENS_CUDA(e, cudaSetDevice(e->device));
    // Time every candidate on the whole ensemble cut short.  Without a complete run each
    // scenario is cut at max_steps.  After one, scenario i is cut at its step count scaled
    // by f = max_steps x (sum of cells) / (sum of cells x steps): the same budget of cell
    // updates, spread as in the real run, so that the few longest scenarios, which set the
    // critical path of the real run, weigh as much in the timing as they will there.
    std::vector<long long> saved(e->n);
    double f = 0.0;
    if (e->have_steps) {
        double c = 0.0, w = 0.0;
        for (int i = 0; i < e->n; i++) {
            const double ci = (double)e->desc[i].rows * e->desc[i].cols;
            c += ci;
            w += ci * (double)e->work_steps[i];
        }
        f = w > 0.0 ? (double)max_steps * c / w : 0.0;
    }
    for (int i = 0; i < e->n; i++) {
        saved[i] = e->host[i].max_steps;
        const long long cap = e->have_steps ? std::llround((double)e->work_steps[i] * f) : (long long)max_steps;
        e->host[i].max_steps = std::min(saved[i], std::max(1LL, cap));
    }
    ENS_CUDA(e, cudaMemcpy(e->dev, e->host.data(), e->n * sizeof(EnsScenario), cudaMemcpyHostToDevice));
    cudaEvent_t a, b;
    ENS_CUDA(e, cudaEventCreate(&a));
    ENS_CUDA(e, cudaEventCreate(&b));
    float best_ms = std::numeric_limits<float>::infinity();
    asx_ensemble_tuning best = e->tuning;
    // the gather kernel's 36 shapes, the strip kernel's 48 (cluster x tile workers per
    // CTA x tile height, or the height chosen per scenario), and 8 split shapes
    std::vector<asx_ensemble_tuning> shapes;
    for (int c : {1, 2, 4, 8}) {
        for (int t : {128, 256, 512})
            for (int k : {1, 2, 4}) shapes.push_back(asx_ensemble_tuning{c, t, k, 0, 0});
        for (int t : {128, 256, 512})
            for (int h : {1, 8, 16, 32}) shapes.push_back(asx_ensemble_tuning{c, t, 1, h, 0});
    }
    // the largest scenarios on whole clusters, the rest on single CTAs
    for (int c : {4, 8})
        for (int sp : {8, 16, 32, 64}) shapes.push_back(asx_ensemble_tuning{c, 256, 1, 1, sp});
    asx_status st = ASX_OK;
    // one untimed launch first (first-launch costs), then the faster of two timings per
    // shape: a single short timing is noisy enough to rank shapes wrongly
    {
        cudaError_t x = reset_state(e, e->stream);
        if (x == cudaSuccess) x = ensure_layout(e, e->tuning);
        if (x == cudaSuccess) x = launch_ensemble(e, e->tuning, e->stream);
        if (x == cudaSuccess) x = cudaStreamSynchronize(e->stream);
        if (x != cudaSuccess) st = efail(e, ASX_ECUDA, std::string("autotune: ") + cudaGetErrorString(x));
    }
    for (size_t si = 0; si < shapes.size() && st == ASX_OK; si++) {
                const asx_ensemble_tuning t = shapes[si];
                if (ensure_layout(e, t) != cudaSuccess) {
                    st = efail(e, ASX_ECUDA, "autotune: layout upload");
                    break;
                }
                float shape_ms = std::numeric_limits<float>::infinity();
                for (int rep = 0; rep < 2 && st == ASX_OK; rep++) {
                    float ms = 0.0f;
                    cudaError_t x = reset_state(e, e->stream);
                    if (x == cudaSuccess) x = cudaEventRecord(a, e->stream);
                    if (x == cudaSuccess) x = launch_ensemble(e, t, e->stream);
                    if (x == cudaSuccess) x = cudaEventRecord(b, e->stream);
                    if (x == cudaSuccess) x = cudaEventSynchronize(b);
                    if (x == cudaSuccess) x = cudaEventElapsedTime(&ms, a, b);
                    if (x != cudaSuccess) {
                        st = efail(e, ASX_ECUDA, std::string("autotune: ") + cudaGetErrorString(x));
                        break;
                    }
                    shape_ms = std::fmin(shape_ms, ms);
                }
                if (st == ASX_OK && shape_ms < best_ms) {
                    best_ms = shape_ms;
                    best = t;
                }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    for (int i = 0; i < e->n; i++) e->host[i].max_steps = saved[i];
    ENS_CUDA(e, cudaMemcpy(e->dev, e->host.data(), e->n * sizeof(EnsScenario), cudaMemcpyHostToDevice));
    if (st) return st;
    e->tuning = best;
    e->tuned = true;
    if (best_out) *best_out = best;
    return ASX_OK;
}

asx_status asx_ensemble_ledger(asx_ensemble *e, int s, asx_ledger *out)
{
    if (!e || !out) return ASX_EINVAL;
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    const EnsScenario &h = e->host[s];
    out->rain_in = h.rain_in;
    out->outflow = h.outflow;
    out->storage = h.storage;
    out->storage0 = h.storage0;
    out->clamped = h.clamped;
    out->steps = h.steps;
    const double scale = std::fmax(h.rain_in, h.storage0);
    const double d = std::fabs(h.storage0 + h.rain_in + h.clamped - h.outflow - h.storage);
    out->defect_rel = scale > 0 ? d / scale : 0.0;
    return ASX_OK;
}

asx_status asx_ensemble_get_fields(asx_ensemble *e, int s, float *h_out, float *v1, float *v2, int kind)
{
    if (!e) return ASX_EINVAL;
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return efail(e, ASX_EINVAL, "bad ptr_kind");
    ENS_CUDA(e, cudaSetDevice(e->device));
    const asx_scenario_desc &d = e->desc[s];
    const EnsScenario &h = e->host[s];
    const int par = h.parity, np = par ^ 1;
    const cudaMemcpyKind mk = kind == ASX_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int pitch = e->pitch[s];
    auto get = [&](void *dst, const void *src) {
        return cudaMemcpy2DAsync(dst, (size_t)d.cols * 4, src, (size_t)pitch * 4, (size_t)d.cols * 4, d.rows, mk,
                                 e->stream);
    };
    if (h_out) {
        ENS_CUDA(e, launch_extract_depth(h.a, par, h.a.mhi[np], e->stream));
        ENS_CUDA(e, get(h_out, h.a.mhi[np]));
    }
    if (v1) ENS_CUDA(e, get(v1, h.a.v1[par]));
    if (v2) ENS_CUDA(e, get(v2, h.a.v2[par]));
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    return ASX_OK;
}

asx_status asx_ensemble_get_state(asx_ensemble *e, int s, float *m_hi, float *m_lo, float *v1, float *v2,
                                  int kind)
{
    if (!e) return ASX_EINVAL;
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return efail(e, ASX_EINVAL, "bad ptr_kind");
    ENS_CUDA(e, cudaSetDevice(e->device));
    const asx_scenario_desc &d = e->desc[s];
    const EnsScenario &h = e->host[s];
    const int par = h.parity;
    const cudaMemcpyKind mk = kind == ASX_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int pitch = e->pitch[s];
    auto get = [&](void *dst, const void *src) {
        return cudaMemcpy2DAsync(dst, (size_t)d.cols * 4, src, (size_t)pitch * 4, (size_t)d.cols * 4, d.rows, mk,
                                 e->stream);
    };
    if (m_hi) ENS_CUDA(e, get(m_hi, h.a.mhi[par]));
    if (m_lo) ENS_CUDA(e, get(m_lo, h.a.mlo[par]));
    if (v1) ENS_CUDA(e, get(v1, h.a.v1[par]));
    if (v2) ENS_CUDA(e, get(v2, h.a.v2[par]));
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    return ASX_OK;
}

asx_status asx_ensemble_get_hydrograph(asx_ensemble *e, int s, double *q, int cap, int *n)
{
    if (!e || !n || cap < 0 || (cap > 0 && !q)) return efail(e, ASX_EINVAL, "bad argument");
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    ENS_CUDA(e, cudaSetDevice(e->device));
    const EnsScenario &h = e->host[s];
    *n = h.n_samples;
    const int m = std::min(h.n_samples, h.max_samples);
    const int k = std::min(m, cap);
    if (k > 0) {
        std::vector<double> cum(k);
        ENS_CUDA(e, cudaMemcpy(cum.data(), h.samples, k * sizeof(double), cudaMemcpyDeviceToHost));
        double prev = 0.0;
        const double sdt = h.sample_dt > 0 ? h.sample_dt : 1.0;
        for (int i = 0; i < k; i++) {
            q[i] = (cum[i] - prev) / sdt;
            prev = cum[i];
        }
    }
    return ASX_OK;
}

asx_status asx_ensemble_get_clock(asx_ensemble *e, int s, double *t, long long *steps)
{
    if (!e) return ASX_EINVAL;
    if (s < 0 || s >= e->n) return efail(e, ASX_EINVAL, "scenario out of range");
    if (t) *t = e->host[s].t;
    if (steps) *steps = e->host[s].steps;
    return ASX_OK;
}

}  // extern "C"
