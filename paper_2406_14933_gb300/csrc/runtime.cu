// runtime.cu -- the C ABI of include/asx.h: raster handles, device memory, field
// upload/download, the device-resident clock, CUDA-graph replay of the step loop and
// the water-budget ledger.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "asx_internal.cuh"

using namespace asx;

namespace asx {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *m, void *base, bool u8, int rows, int cols, int pitch, int box_x, int box_y)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const size_t es = u8 ? 1 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, u8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// 2-D tensor map over a pitched rows x cols plane; out-of-range elements read as zero.
bool make_tensor_map_2d(CUtensorMap *m, void *base, bool u8, int rows, int cols, int pitch, int box_x, int box_y)
{
    return make_map(m, base, u8, rows, cols, pitch, box_x, box_y);
}

bool make_tensor_map_bf16(CUtensorMap *m, const void *base, long long rows, long long cols, long long ld, int box_x,
                          int box_y)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_strip_maps(StripMaps &m, const StepArgs &a, int rows, int cols, int pitch)
{
    bool ok = true;
    const int bf = kStripW + 8;
    for (int p = 0; p < 2; p++) {
        ok = ok && make_map(&m.mhi[p], a.mhi[p], false, rows, cols, pitch, bf, kStripChunkRows);
        ok = ok && make_map(&m.v1[p], a.v1[p], false, rows, cols, pitch, bf, kStripChunkRows);
        ok = ok && make_map(&m.v2[p], a.v2[p], false, rows, cols, pitch, bf, kStripChunkRows);
        ok = ok && make_map(&m.mlo[p], a.mlo[p], false, rows, cols, pitch, kStripW, kStripChunkRows);
    }
    ok = ok && make_map(&m.z, (void *)a.z, false, rows, cols, pitch, bf, kStripChunkRows);
    if (a.cls)
        ok = ok && make_map(&m.th, (void *)a.cls, true, rows, cols, pitch, kStripW + 16, kStripChunkRows);
    else
        ok = ok && make_map(&m.th, (void *)a.theta, false, rows, cols, pitch, bf, kStripChunkRows);
    return ok;
}

}  // namespace asx

namespace {

constexpr int kGraphSteps = 32;   // step launches captured in one graph
constexpr int kTileRowsDefault = 32;

enum StepVariant { kVariantStrip = 0, kVariantGather = 1, kVariantFp64 = 2 };

// Step kernel variant: ASX_STEP_KERNEL=gather selects the one-thread-per-cell gather
// kernel; the default is the TMA strip kernel.  ASX_TILE_ROWS sets the strip tile height.
int variant_from_env()
{
    const char *v = std::getenv("ASX_STEP_KERNEL");
    if (v && std::strcmp(v, "gather") == 0) return kVariantGather;
    return kVariantStrip;
}

int tile_rows_from_env()
{
    const char *v = std::getenv("ASX_TILE_ROWS");
    int t = v ? std::atoi(v) : kTileRowsDefault;
    if (t < 2) t = 2;
    if (t > 1024) t = 1024;
    return t;
}

// Leading part of DevCtl that the host reads after a call (the clock and flags).
constexpr size_t kCtlHead = offsetof(DevCtl, cmax_bits);

}  // namespace

struct asx_raster {
    asx_raster_desc desc{};
    cudaStream_t stream = nullptr;
    int rows = 0, cols = 0, pitch = 0;
    size_t plane = 0;                   // bytes of one pitched float32 field
    float *buf = nullptr;               // all float planes in one allocation
    uint8_t *cls = nullptr;
    DevCtl *ctl = nullptr;
    double *samples = nullptr;
    double *scan_parts = nullptr;
    int scan_n = 0;
    StepArgs args{};
    StepArgs64 a64{};                   // FP64 mode (desc.precision == ASX_FP64)
    bool fp64 = false;
    int variant = kVariantStrip;
    StripMaps maps{};
    DevCtl host_ctl{};                  // parameter image (device copy is authoritative)
    DevCtl *mirror = nullptr;           // pinned host copies of the control head [2]
    bool have_params = false, have_fields = false;
    cudaGraphExec_t graph = nullptr;
    std::string err;
};

namespace {

asx_status fail(asx_raster *r, asx_status st, const std::string &msg)
{
    if (r) r->err = msg;
    return st;
}

#define ASX_CUDA(r, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((r), ASX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
bool finite_host(const T *p, size_t n)
{
    for (size_t i = 0; i < n; i++)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Copies a dense rows x cols field (host or device) into a pitched device plane.
cudaError_t put_plane(asx_raster *r, void *dst, const void *src, size_t esize, int kind)
{
    return cudaMemcpy2DAsync(dst, (size_t)r->pitch * esize, src, (size_t)r->cols * esize,
                             (size_t)r->cols * esize, (size_t)r->rows,
                             kind == ASX_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             r->stream);
}

cudaError_t get_plane(asx_raster *r, void *dst, const void *src, size_t esize, int kind)
{
    return cudaMemcpy2DAsync(dst, (size_t)r->cols * esize, src, (size_t)r->pitch * esize,
                             (size_t)r->cols * esize, (size_t)r->rows,
                             kind == ASX_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             r->stream);
}

asx_status set_device(asx_raster *r)
{
    ASX_CUDA(r, cudaSetDevice(r->desc.device));
    return ASX_OK;
}

// Storage and c_max of the current state (the float32 or the float64 scan).
cudaError_t scan_state(asx_raster *r, int set_storage0)
{
    if (r->fp64) return launch_scan64(r->a64, r->scan_parts, r->scan_n, set_storage0, r->stream);
    return launch_scan(r->args, r->scan_parts, r->scan_n, set_storage0, r->stream);
}

// Reads the control head (clock, flags) into mirror[0]; synchronises the stream.
asx_status read_head(asx_raster *r, DevCtl **out)
{
    ASX_CUDA(r, cudaMemcpyAsync(r->mirror, r->ctl, kCtlHead, cudaMemcpyDeviceToHost, r->stream));
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    *out = r->mirror;
    return ASX_OK;
}

template <typename T>
cudaError_t put_ctl_field(asx_raster *r, T DevCtl::*field, const T &value)
{
    const size_t off = reinterpret_cast<size_t>(&(reinterpret_cast<DevCtl *>(0)->*field));
    return cudaMemcpyAsync(reinterpret_cast<char *>(r->ctl) + off, &value, sizeof(T),
                           cudaMemcpyHostToDevice, r->stream);
}

void drop_graph(asx_raster *r)
{
    if (r->graph) {
        cudaGraphExecDestroy(r->graph);
        r->graph = nullptr;
    }
}

cudaError_t launch_step(asx_raster *r, cudaStream_t s)
{
    if (r->variant == kVariantFp64) return launch_step_fp64(r->a64, s);
    if (r->variant == kVariantGather) return launch_step_gather(r->args, s);
    return launch_step_strip(r->args, r->maps, s);
}

asx_status build_graph(asx_raster *r)
{
    if (r->graph) return ASX_OK;
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    // capture on a private stream so the caller's stream (possibly the legacy default
    // stream, which cannot be captured) is never put in capture mode
    ASX_CUDA(r, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; i++) e = launch_step(r, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        r->graph = nullptr;
        return fail(r, ASX_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    return ASX_OK;
}

asx_status check_numeric(asx_raster *r, const DevCtl *h)
{
    if (h->err & kErrNumeric)
        return fail(r, ASX_ENUMERIC, "the state became non-finite at step " + std::to_string(h->step));
    if (h->err & kErrTimeout) return fail(r, ASX_ETIMEOUT, "a bounded wait in a kernel ran out");
    if (h->err & kErrBounds) return fail(r, ASX_EBOUNDS, "an index outside its buffer (bounds-checked build)");
    return ASX_OK;
}

// Replays the step graph until the device clock reports no pending step.  Keeps two
// graphs in flight and polls the clock copied after the older one, so the GPU does not
// idle while the host checks; kernels launched past the target are no-ops.
asx_status drive(asx_raster *r)
{
    asx_status st = build_graph(r);
    if (st) return st;
    cudaEvent_t ev[2];
    ASX_CUDA(r, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    cudaError_t e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(r, ASX_ECUDA, std::string("event: ") + cudaGetErrorString(e));
    }
    for (long long k = 0;; k++) {
        const int j = (int)(k & 1);
        e = cudaGraphLaunch(r->graph, r->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&r->mirror[j], r->ctl, kCtlHead, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[j], r->stream);
        if (e == cudaSuccess && k >= 1) e = cudaEventSynchronize(ev[j ^ 1]);
        if (e != cudaSuccess) break;
        if (k >= 1) {
            const DevCtl *h = &r->mirror[j ^ 1];
            if (!h->active || h->err) break;
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(r->stream);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(r, ASX_ECUDA, std::string("step graph: ") + cudaGetErrorString(e));
    return ASX_OK;
}

}  // namespace

extern "C" {

const char *asx_last_error(const asx_raster *r)
{
    if (!r) return "null raster handle";
    return r->err.c_str();
}

asx_status asx_create_raster(const asx_raster_desc *desc, asx_raster **out)
{
    if (!desc || !out) return ASX_EINVAL;
    *out = nullptr;
    if (desc->rows < 2 || desc->cols < 2 || !(desc->edge_m > 0.0) || !std::isfinite(desc->edge_m))
        return ASX_EINVAL;
    if ((long long)desc->rows * desc->cols >= (1LL << 31)) return ASX_EINVAL;
    for (int s = 0; s < 4; s++) {
        if (desc->bc[s] < ASX_BC_WALL || desc->bc[s] > ASX_BC_DIRICHLET) return ASX_EINVAL;
        if (desc->free_begin[s] < 0 || desc->free_end[s] < desc->free_begin[s]) return ASX_EINVAL;
    }
    if (desc->n_classes < 0 || desc->n_classes > kMaxClasses || desc->max_samples < 0) return ASX_EINVAL;
    if (desc->precision != ASX_FP32_COMP && desc->precision != ASX_FP64) return ASX_EINVAL;

    asx_raster *r = new (std::nothrow) asx_raster();
    if (!r) return ASX_ENOMEM;
    r->desc = *desc;
    r->stream = (cudaStream_t)desc->cuda_stream;
    r->rows = desc->rows;
    r->cols = desc->cols;
    r->pitch = (desc->cols + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
    r->fp64 = desc->precision == ASX_FP64;
    // FP64 mode: every plane holds float64 (the state's six planes, bed, porosity)
    r->plane = (size_t)r->rows * r->pitch * (r->fp64 ? sizeof(double) : sizeof(float));
    asx_status st = set_device(r);
    if (st) { delete r; return st; }
    // planes: 2 x (mhi, mlo, v1, v2), z, theta
    const int nplanes = 8 + 1 + (desc->n_classes == 0 ? 1 : 0);
    cudaError_t e = cudaMalloc(&r->buf, r->plane * nplanes);
    if (e == cudaSuccess && desc->n_classes > 0) e = cudaMalloc(&r->cls, (size_t)r->rows * r->pitch);
    if (e == cudaSuccess) e = cudaMalloc(&r->ctl, sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMalloc(&r->samples, sizeof(double) * (size_t)(desc->max_samples > 0 ? desc->max_samples : 1));
    r->scan_n = scan_blocks(r->rows, r->cols);
    if (e == cudaSuccess) e = cudaMalloc(&r->scan_parts, sizeof(double) * 2 * (size_t)r->scan_n);
    if (e == cudaSuccess) e = cudaMallocHost(&r->mirror, 2 * sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMemsetAsync(r->buf, 0, r->plane * nplanes, r->stream);
    if (e != cudaSuccess) {
        asx_destroy_raster(r);
        return e == cudaErrorMemoryAllocation ? ASX_ENOMEM : ASX_ECUDA;
    }
    StepArgs &a = r->args;
    a.rows = r->rows;
    a.cols = r->cols;
    a.pitch = r->pitch;
    r->variant = r->fp64 ? kVariantFp64 : variant_from_env();
    a.tile_rows = tile_rows_from_env();
    if (r->variant == kVariantGather) a.nblocks = step_gather_blocks(r->rows, r->cols);
    else if (r->variant == kVariantStrip) step_strip_layout(a);
    const size_t pe = r->plane / sizeof(float);
    for (int p = 0; p < 2; p++) {
        a.mhi[p] = r->buf + (size_t)(4 * p + 0) * pe;
        a.mlo[p] = r->buf + (size_t)(4 * p + 1) * pe;
        a.v1[p] = r->buf + (size_t)(4 * p + 2) * pe;
        a.v2[p] = r->buf + (size_t)(4 * p + 3) * pe;
    }
    a.z = r->buf + 8 * pe;
    a.theta = desc->n_classes == 0 ? r->buf + 9 * pe : nullptr;
    a.cls = r->cls;
    for (int s = 0; s < 4; s++) {
        a.bc[s] = desc->bc[s];
        a.fb[s] = desc->free_begin[s];
        a.fe[s] = desc->free_end[s];
    }
    a.ctl = r->ctl;
    if (r->fp64) {
        // the same plane slots, counted in float64 elements (rows x pitch each)
        StepArgs64 &b = r->a64;
        double *dbuf = reinterpret_cast<double *>(r->buf);
        const size_t pd = r->plane / sizeof(double);
        b.rows = r->rows;
        b.cols = r->cols;
        b.pitch = r->pitch;
        for (int p = 0; p < 2; p++) {
            b.m[p] = dbuf + (size_t)(4 * p + 0) * pd;
            b.v1[p] = dbuf + (size_t)(4 * p + 2) * pd;
            b.v2[p] = dbuf + (size_t)(4 * p + 3) * pd;
        }
        b.z = dbuf + 8 * pd;
        b.theta = desc->n_classes == 0 ? dbuf + 9 * pd : nullptr;
        b.cls = r->cls;
        for (int s = 0; s < 4; s++) {
            b.bc[s] = desc->bc[s];
            b.fb[s] = desc->free_begin[s];
            b.fe[s] = desc->free_end[s];
        }
        b.nblocks = step_fp64_blocks(r->rows, r->cols);
        b.ctl = r->ctl;
    }
    if (r->variant == kVariantStrip) {
        const bool ok = make_strip_maps(r->maps, a, r->rows, r->cols, r->pitch);
        if (!ok || step_strip_configure() != cudaSuccess) {
            asx_destroy_raster(r);
            return ASX_ECUDA;
        }
    }
    DevCtl &c = r->host_ctl;
    std::memset(&c, 0, sizeof(DevCtl));
    c.t_end = std::numeric_limits<double>::infinity();
    c.max_samples = desc->max_samples;
    c.samples = r->samples;
    c.sigma = 1.5 * std::sqrt(3.0) * desc->edge_m * desc->edge_m;
    c.phi = c.sigma / (6.0 * desc->edge_m);
    c.ncells = (long long)r->rows * r->cols;
    c.fp64 = r->fp64 ? 1 : 0;
    e = cudaMemcpyAsync(r->ctl, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) {
        asx_destroy_raster(r);
        return ASX_ECUDA;
    }
    *out = r;
    return ASX_OK;
}

asx_status asx_destroy_raster(asx_raster *r)
{
    if (!r) return ASX_OK;
    cudaSetDevice(r->desc.device);
    if (r->stream) cudaStreamSynchronize(r->stream);
    drop_graph(r);
    cudaFree(r->buf);
    cudaFree(r->cls);
    cudaFree(r->ctl);
    cudaFree(r->samples);
    cudaFree(r->scan_parts);
    if (r->mirror) cudaFreeHost(r->mirror);
    delete r;
    return ASX_OK;
}

asx_status asx_set_params(asx_raster *r, const asx_params *p)
{
    if (!r || !p) return fail(r, ASX_EINVAL, "null argument");
    if (!(p->g > 0) || !std::isfinite(p->g)) return fail(r, ASX_EINVAL, "g must be > 0");
    if (!(p->cfl > 0) || !(p->cfl <= 1)) return fail(r, ASX_EINVAL, "cfl must be in (0, 1]");
    if (!(p->dt_max > 0) || !std::isfinite(p->dt_max)) return fail(r, ASX_EINVAL, "dt_max must be > 0");
    if (!(p->sample_dt >= 0) || !std::isfinite(p->sample_dt)) return fail(r, ASX_EINVAL, "sample_dt must be >= 0");
    if (p->n_rain < 0 || p->n_rain > kMaxRain) return fail(r, ASX_EINVAL, "n_rain out of range");
    if (p->viscosity != 0 && p->viscosity != 1) return fail(r, ASX_EINVAL, "viscosity must be 0 or 1");
    if (!(p->tau >= 0) || !std::isfinite(p->tau)) return fail(r, ASX_EINVAL, "tau must be >= 0");
    if (!(p->h_dry >= 0) || !std::isfinite(p->h_dry)) return fail(r, ASX_EINVAL, "h_dry must be >= 0");
    for (int s = 0; s < 4; s++)
        if (!(p->bc_q[s] >= 0) || !std::isfinite(p->bc_q[s]) || !(p->bc_h[s] >= 0) || !std::isfinite(p->bc_h[s]) ||
            !std::isfinite(p->bc_u[s]))
            return fail(r, ASX_EINVAL, "boundary values out of range (bc_q, bc_h >= 0, finite)");
    if (p->n_rain > 0 && (!p->rain_t || !p->rain_r)) return fail(r, ASX_EINVAL, "rain table missing");
    for (int k = 0; k < p->n_rain; k++) {
        if (!std::isfinite(p->rain_t[k]) || !std::isfinite(p->rain_r[k]) || p->rain_r[k] < 0)
            return fail(r, ASX_EINVAL, "rain table value out of range");
        if (k > 0 && p->rain_t[k] < p->rain_t[k - 1]) return fail(r, ASX_EINVAL, "rain times must increase");
    }
    StepArgs &a = r->args;
    const int nc = r->desc.n_classes;
    if (nc == 0) {
        if (!(p->alpha_s >= 0) || !(p->alpha_p >= 0) || !std::isfinite(p->alpha_s) || !std::isfinite(p->alpha_p))
            return fail(r, ASX_EINVAL, "alpha_s, alpha_p must be >= 0");
        a.alpha_s = (float)p->alpha_s;
        a.alpha_p = (float)p->alpha_p;
    } else {
        if (!p->class_theta || !p->class_alpha_p || !p->class_alpha_s)
            return fail(r, ASX_EINVAL, "class tables missing");
        for (int k = 0; k < nc; k++) {
            const float th = p->class_theta[k], ap = p->class_alpha_p[k], as = p->class_alpha_s[k];
            if (!(th > 0) || !(th <= 1) || !(ap >= 0) || !(as >= 0) || !std::isfinite(ap) || !std::isfinite(as))
                return fail(r, ASX_EINVAL, "class table value out of range");
            a.cls_theta[k] = th;
            a.cls_rth[k] = (float)(1.0 / (double)th);
            a.cls_a[k] = ap * (1.0f - th);
            a.cls_b[k] = th * as;
        }
    }
    const double l = r->desc.edge_m;
    a.l = (float)l;
    a.g = (float)p->g;
    a.visc = p->viscosity;
    a.tau = (float)p->tau;
    a.h_dry = (float)p->h_dry;
    for (int s = 0; s < 4; s++) {
        a.bq[s] = (float)p->bc_q[s];
        a.bhc[s] = (float)std::cbrt(p->bc_q[s] * p->bc_q[s] / p->g);
        a.bh[s] = (float)p->bc_h[s];
        a.bu[s] = (float)p->bc_u[s];
    }
    {
        StepArgs64 &b = r->a64;
        if (nc == 0) {
            b.alpha_s = p->alpha_s;
            b.alpha_p = p->alpha_p;
        } else {
            for (int k = 0; k < nc; k++) {
                b.cls_theta[k] = (double)p->class_theta[k];
                b.cls_as[k] = (double)p->class_alpha_s[k];
                b.cls_ap[k] = (double)p->class_alpha_p[k];
            }
        }
        b.l = l;
        b.g = p->g;
        b.tau = p->tau;
        b.h_dry = p->h_dry;
        b.visc = p->viscosity;
        for (int s = 0; s < 4; s++) {
            b.bq[s] = p->bc_q[s];
            b.bh[s] = p->bc_h[s];
            b.bu[s] = p->bc_u[s];
        }
    }
    const double s3 = std::sqrt(3.0) / 2.0;
    const double n1[3] = {1.0, 0.5, -0.5}, n2[3] = {0.0, s3, s3};
    for (int d = 0; d < 3; d++) {
        a.cpe[d][0] = (float)(-0.5 * l * p->g * n1[d]);
        a.cpe[d][1] = (float)(-0.5 * l * p->g * n2[d]);
        a.cpm[d][0] = (float)(-4.0 * p->g * n1[d]);
        a.cpm[d][1] = (float)(-4.0 * p->g * n2[d]);
    }
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl &c = r->host_ctl;
    c.g = p->g;
    c.cfl = p->cfl;
    c.dt_max = p->dt_max;
    c.sample_dt = p->sample_dt;
    c.n_rain = p->n_rain;
    for (int k = 0; k < p->n_rain; k++) {
        c.rain_t[k] = p->rain_t[k];
        c.rain_r[k] = p->rain_r[k];
    }
    // parameters live at the end of DevCtl: copy that tail only
    ASX_CUDA(r, cudaMemcpyAsync(reinterpret_cast<char *>(r->ctl) + offsetof(DevCtl, g),
                                reinterpret_cast<char *>(&c) + offsetof(DevCtl, g),
                                sizeof(DevCtl) - offsetof(DevCtl, g), cudaMemcpyHostToDevice, r->stream));
    ASX_CUDA(r, put_ctl_field(r, &DevCtl::sample_dt, c.sample_dt));
    drop_graph(r);
    r->have_params = true;
    if (r->have_fields) {
        ASX_CUDA(r, launch_prepare(r->ctl, kPrepRecompute, 0.0, 0, r->stream));
    }
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    return ASX_OK;
}

asx_status asx_set_fields(asx_raster *r, const double *z, const float *theta, const uint8_t *cls,
                          const float *h0, const float *v1, const float *v2, int kind)
{
    if (!r) return ASX_EINVAL;
    if (!r->have_params) return fail(r, ASX_ESTATE, "asx_set_params must come first");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return fail(r, ASX_EINVAL, "bad ptr_kind");
    const int nc = r->desc.n_classes;
    if (!z || !h0) return fail(r, ASX_EINVAL, "z and h0 are required");
    if (nc == 0 && (!theta || cls)) return fail(r, ASX_EINVAL, "per-cell porosity expected");
    if (nc > 0 && (!cls || theta)) return fail(r, ASX_EINVAL, "per-cell class expected");
    const size_t n = (size_t)r->rows * r->cols;
    if (kind == ASX_PTR_HOST) {
        if (!finite_host(z, n)) return fail(r, ASX_EINVAL, "z has a non-finite value");
        for (size_t i = 0; i < n; i++)
            if (!(h0[i] >= 0.0f) || !std::isfinite(h0[i])) return fail(r, ASX_EINVAL, "h0 must be finite and >= 0");
        if (v1 && !finite_host(v1, n)) return fail(r, ASX_EINVAL, "v1 has a non-finite value");
        if (v2 && !finite_host(v2, n)) return fail(r, ASX_EINVAL, "v2 has a non-finite value");
        if (theta)
            for (size_t i = 0; i < n; i++)
                if (!(theta[i] > 0.0f) || !(theta[i] <= 1.0f)) return fail(r, ASX_EINVAL, "theta must be in (0, 1]");
        if (cls)
            for (size_t i = 0; i < n; i++)
                if (cls[i] >= nc) return fail(r, ASX_EINVAL, "class id out of range");
    }
    asx_status st = set_device(r);
    if (st) return st;
    StepArgs &a = r->args;
    if (cls) ASX_CUDA(r, put_plane(r, (void *)a.cls, cls, 1, kind));
    if (r->fp64) {
        // float64 planes: the bed as given; porosity, depth and velocities widened from
        // float32 staged (float32, pitched) in the parity-1 planes
        StepArgs64 &b = r->a64;
        ASX_CUDA(r, put_plane(r, (void *)b.z, z, sizeof(double), kind));
        float *st_h = reinterpret_cast<float *>(b.m[1]), *st_1 = reinterpret_cast<float *>(b.v1[1]);
        float *st_2 = reinterpret_cast<float *>(b.v2[1]);
        if (theta) {
            ASX_CUDA(r, put_plane(r, st_h, theta, sizeof(float), kind));
            ASX_CUDA(r, launch_widen(st_h, r->rows, r->cols, r->pitch, (double *)b.theta, r->pitch, r->stream));
        }
        ASX_CUDA(r, put_plane(r, st_h, h0, sizeof(float), kind));
        if (v1) ASX_CUDA(r, put_plane(r, st_1, v1, sizeof(float), kind));
        if (v2) ASX_CUDA(r, put_plane(r, st_2, v2, sizeof(float), kind));
        ASX_CUDA(r, launch_init64(b, 0, st_h, v1 ? st_1 : nullptr, v2 ? st_2 : nullptr, r->stream));
    } else {
        // the bed rounded to the nearest float32
        if (kind == ASX_PTR_HOST) {
            std::vector<float> zf(n);
            for (size_t i = 0; i < n; i++) zf[i] = (float)z[i];
            ASX_CUDA(r, put_plane(r, (void *)a.z, zf.data(), sizeof(float), kind));
            ASX_CUDA(r, cudaStreamSynchronize(r->stream));     // zf is released on return
        } else {
            ASX_CUDA(r, launch_narrow(z, r->rows, r->cols, r->cols, (float *)a.z, r->pitch, r->stream));
        }
        if (theta) ASX_CUDA(r, put_plane(r, (void *)a.theta, theta, sizeof(float), kind));
        // stage h0, v in the parity-1 planes, convert into parity 0
        ASX_CUDA(r, put_plane(r, a.mhi[1], h0, sizeof(float), kind));
        if (v1) ASX_CUDA(r, put_plane(r, a.v1[1], v1, sizeof(float), kind));
        if (v2) ASX_CUDA(r, put_plane(r, a.v2[1], v2, sizeof(float), kind));
        ASX_CUDA(r, launch_init_state(a, 0, a.mhi[1], v1 ? a.v1[1] : nullptr, v2 ? a.v2[1] : nullptr, r->stream));
    }
    // reset clock and ledger (everything before the parameters)
    DevCtl &c = r->host_ctl;
    c.t = 0.0;
    c.dt = 0.0;
    c.t_next = 0.0;
    c.t_end = std::numeric_limits<double>::infinity();
    c.step = 0;
    c.step_limit = 0;
    c.active = 0;
    c.parity = 0;
    c.err = 0;
    c.cmax_bits = 0;
    c.cmax64_bits = 0ull;
    c.done_ctas = 0;
    c.scan_done = 0;
    c.out_fx[0] = c.out_fx[1] = c.clamp_fx[0] = c.clamp_fx[1] = 0ull;
    c.rain_in = c.outflow = c.clamped = c.storage0 = c.storage = 0.0;
    c.n_samples = 0;
    ASX_CUDA(r, cudaMemcpyAsync(r->ctl, &c, offsetof(DevCtl, g), cudaMemcpyHostToDevice, r->stream));
    ASX_CUDA(r, scan_state(r, 1));
    ASX_CUDA(r, launch_prepare(r->ctl, kPrepRecompute, 0.0, 0, r->stream));
    DevCtl *h;
    st = read_head(r, &h);
    if (st) return st;
    r->have_fields = true;
    return check_numeric(r, h);
}

asx_status asx_step(asx_raster *r, int n_steps, double *t_out)
{
    if (!r) return ASX_EINVAL;
    if (n_steps < 0) return fail(r, ASX_EINVAL, "n_steps must be >= 0");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    ASX_CUDA(r, launch_prepare(r->ctl, kPrepSteps, 0.0, n_steps, r->stream));
    if (n_steps < kGraphSteps) {
        for (int i = 0; i < n_steps; i++) ASX_CUDA(r, launch_step(r, r->stream));
    } else {
        st = build_graph(r);
        if (st) return st;
        const int full = n_steps / kGraphSteps;
        for (int i = 0; i < full; i++) ASX_CUDA(r, cudaGraphLaunch(r->graph, r->stream));
        for (int i = 0; i < n_steps - full * kGraphSteps; i++)
            ASX_CUDA(r, launch_step(r, r->stream));
    }
    DevCtl *h;
    st = read_head(r, &h);
    if (st) return st;
    if (t_out) *t_out = h->t;
    return check_numeric(r, h);
}

asx_status asx_run_until(asx_raster *r, double t_end, double *t_out)
{
    if (!r) return ASX_EINVAL;
    if (!std::isfinite(t_end)) return fail(r, ASX_EINVAL, "t_end must be finite");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    ASX_CUDA(r, launch_prepare(r->ctl, kPrepUntil, t_end, 0, r->stream));
    DevCtl *h;
    st = read_head(r, &h);
    if (st) return st;
    if (h->active) {
        st = drive(r);
        if (st) return st;
        st = read_head(r, &h);
        if (st) return st;
    }
    if (t_out) *t_out = h->t;
    return check_numeric(r, h);
}

asx_status asx_mass_ledger(asx_raster *r, int scenario, asx_ledger *out)
{
    if (!r || !out) return fail(r, ASX_EINVAL, "null argument");
    if (scenario != 0) return fail(r, ASX_EINVAL, "scenario must be 0 for a single raster");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    ASX_CUDA(r, scan_state(r, 0));
    // scan also refreshes c_max of the current state, which equals what the last step
    // recorded; the pending dt is unchanged
    DevCtl *c = &r->mirror[1];
    ASX_CUDA(r, cudaMemcpyAsync(c, r->ctl, offsetof(DevCtl, sample_dt), cudaMemcpyDeviceToHost, r->stream));
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    out->rain_in = c->rain_in;
    out->outflow = c->outflow;
    out->storage = c->storage;
    out->storage0 = c->storage0;
    out->clamped = c->clamped;
    out->steps = c->step;
    const double scale = std::fmax(c->rain_in, c->storage0);
    const double d = std::fabs(c->storage0 + c->rain_in + c->clamped - c->outflow - c->storage);
    out->defect_rel = scale > 0 ? d / scale : 0.0;
    return ASX_OK;
}

asx_status asx_get_fields(asx_raster *r, int scenario, float *h, float *v1, float *v2, int kind)
{
    if (!r) return ASX_EINVAL;
    if (scenario != 0) return fail(r, ASX_EINVAL, "scenario must be 0 for a single raster");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return fail(r, ASX_EINVAL, "bad ptr_kind");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl *hd;
    st = read_head(r, &hd);
    if (st) return st;
    const int par = hd->parity, np = par ^ 1;
    const StepArgs &a = r->args;
    if (r->fp64) {
        // float32 copies of h, v1, v2 in the other parity's planes (free between steps)
        const StepArgs64 &b = r->a64;
        float *h32 = reinterpret_cast<float *>(b.m[np]), *u32 = reinterpret_cast<float *>(b.v1[np]);
        float *w32 = reinterpret_cast<float *>(b.v2[np]);
        ASX_CUDA(r, launch_extract64(b, par, nullptr, nullptr, nullptr, h32, u32, w32, r->stream));
        if (h) ASX_CUDA(r, get_plane(r, h, h32, sizeof(float), kind));
        if (v1) ASX_CUDA(r, get_plane(r, v1, u32, sizeof(float), kind));
        if (v2) ASX_CUDA(r, get_plane(r, v2, w32, sizeof(float), kind));
        ASX_CUDA(r, cudaStreamSynchronize(r->stream));
        return ASX_OK;
    }
    if (h) {
        ASX_CUDA(r, launch_extract_depth(a, par, a.mhi[np], r->stream));
        ASX_CUDA(r, get_plane(r, h, a.mhi[np], sizeof(float), kind));
    }
    if (v1) ASX_CUDA(r, get_plane(r, v1, a.v1[par], sizeof(float), kind));
    if (v2) ASX_CUDA(r, get_plane(r, v2, a.v2[par], sizeof(float), kind));
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    return ASX_OK;
}

asx_status asx_get_fields64(asx_raster *r, int scenario, double *h, double *v1, double *v2, int kind)
{
    if (!r) return ASX_EINVAL;
    if (scenario != 0) return fail(r, ASX_EINVAL, "scenario must be 0 for a single raster");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return fail(r, ASX_EINVAL, "bad ptr_kind");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl *hd;
    st = read_head(r, &hd);
    if (st) return st;
    const int par = hd->parity;
    // three pitched float64 planes of scratch for the duration of the call
    double *tmp = nullptr;
    const size_t pl = (size_t)r->rows * r->pitch;
    ASX_CUDA(r, cudaMalloc(&tmp, 3 * pl * sizeof(double)));
    cudaError_t e;
    if (r->fp64) e = launch_extract64(r->a64, par, tmp, tmp + pl, tmp + 2 * pl, nullptr, nullptr, nullptr, r->stream);
    else e = launch_extract_wide(r->args, par, tmp, tmp + pl, tmp + 2 * pl, r->stream);
    if (e == cudaSuccess && h) e = get_plane(r, h, tmp, sizeof(double), kind);
    if (e == cudaSuccess && v1) e = get_plane(r, v1, tmp + pl, sizeof(double), kind);
    if (e == cudaSuccess && v2) e = get_plane(r, v2, tmp + 2 * pl, sizeof(double), kind);
    cudaError_t e2 = cudaStreamSynchronize(r->stream);
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(r, ASX_ECUDA, std::string("get_fields64: ") + cudaGetErrorString(e));
    return ASX_OK;
}

asx_status asx_get_state(asx_raster *r, float *mhi, float *mlo, float *v1, float *v2, int kind)
{
    if (!r) return ASX_EINVAL;
    if (r->fp64) return fail(r, ASX_EINVAL, "the compensated float32 state does not exist in FP64 mode");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return fail(r, ASX_EINVAL, "bad ptr_kind");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl *hd;
    st = read_head(r, &hd);
    if (st) return st;
    const int par = hd->parity;
    const StepArgs &a = r->args;
    if (mhi) ASX_CUDA(r, get_plane(r, mhi, a.mhi[par], sizeof(float), kind));
    if (mlo) ASX_CUDA(r, get_plane(r, mlo, a.mlo[par], sizeof(float), kind));
    if (v1) ASX_CUDA(r, get_plane(r, v1, a.v1[par], sizeof(float), kind));
    if (v2) ASX_CUDA(r, get_plane(r, v2, a.v2[par], sizeof(float), kind));
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    return ASX_OK;
}

asx_status asx_set_state(asx_raster *r, const float *mhi, const float *mlo, const float *v1,
                         const float *v2, int kind, double t, long long step,
                         const asx_ledger *ledger, int n_samples, const double *samples)
{
    if (!r) return ASX_EINVAL;
    if (r->fp64) return fail(r, ASX_EINVAL, "the compensated float32 state does not exist in FP64 mode");
    if (!mhi || !mlo || !v1 || !v2 || !ledger) return fail(r, ASX_EINVAL, "null argument");
    if (kind != ASX_PTR_HOST && kind != ASX_PTR_DEVICE) return fail(r, ASX_EINVAL, "bad ptr_kind");
    if (!r->have_fields) return fail(r, ASX_ESTATE, "asx_set_fields must come first");
    if (!std::isfinite(t) || step < 0 || n_samples < 0 || (n_samples > 0 && !samples))
        return fail(r, ASX_EINVAL, "bad clock");
    // the hydrograph samples recorded by time t: the steps are cut at every sample time,
    // so n_samples sample times lie at or before t and the next one after it
    const double sdt = r->host_ctl.sample_dt;
    if (sdt > 0.0 && !((double)n_samples * sdt <= t && t < (double)(n_samples + 1) * sdt))
        return fail(r, ASX_EINVAL, "n_samples does not match t: the sample times up to t must all be recorded");
    asx_status st = set_device(r);
    if (st) return st;
    const StepArgs &a = r->args;
    ASX_CUDA(r, put_plane(r, a.mhi[0], mhi, sizeof(float), kind));
    ASX_CUDA(r, put_plane(r, a.mlo[0], mlo, sizeof(float), kind));
    ASX_CUDA(r, put_plane(r, a.v1[0], v1, sizeof(float), kind));
    ASX_CUDA(r, put_plane(r, a.v2[0], v2, sizeof(float), kind));
    const int ns = n_samples < r->desc.max_samples ? n_samples : r->desc.max_samples;
    if (ns > 0)
        ASX_CUDA(r, cudaMemcpyAsync(r->samples, samples, sizeof(double) * ns, cudaMemcpyHostToDevice, r->stream));
    DevCtl &c = r->host_ctl;
    c.t = t;
    c.dt = 0.0;
    c.t_next = t;
    c.t_end = std::numeric_limits<double>::infinity();
    c.step = step;
    c.step_limit = step;
    c.active = 0;
    c.parity = 0;
    c.err = 0;
    c.cmax_bits = 0;
    c.done_ctas = 0;
    c.scan_done = 0;
    c.out_fx[0] = c.out_fx[1] = c.clamp_fx[0] = c.clamp_fx[1] = 0ull;
    c.rain_in = ledger->rain_in;
    c.outflow = ledger->outflow;
    c.clamped = ledger->clamped;
    c.storage0 = ledger->storage0;
    c.storage = ledger->storage;
    c.n_samples = n_samples;
    ASX_CUDA(r, cudaMemcpyAsync(r->ctl, &c, offsetof(DevCtl, g), cudaMemcpyHostToDevice, r->stream));
    ASX_CUDA(r, scan_state(r, 0));
    ASX_CUDA(r, put_ctl_field(r, &DevCtl::storage0, ledger->storage0));
    ASX_CUDA(r, launch_prepare(r->ctl, kPrepRecompute, 0.0, 0, r->stream));
    DevCtl *h;
    st = read_head(r, &h);
    if (st) return st;
    return check_numeric(r, h);
}

asx_status asx_get_hydrograph(asx_raster *r, int scenario, double *q, int cap, int *n)
{
    if (!r || !n || cap < 0 || (cap > 0 && !q)) return fail(r, ASX_EINVAL, "bad argument");
    if (scenario != 0) return fail(r, ASX_EINVAL, "scenario must be 0 for a single raster");
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl *c = &r->mirror[1];
    ASX_CUDA(r, cudaMemcpyAsync(c, r->ctl, offsetof(DevCtl, g), cudaMemcpyDeviceToHost, r->stream));
    ASX_CUDA(r, cudaStreamSynchronize(r->stream));
    const int ns = c->n_samples;
    const double sdt = c->sample_dt > 0 ? c->sample_dt : 1.0;
    *n = ns;
    const int m = ns < r->desc.max_samples ? ns : r->desc.max_samples;
    const int k = m < cap ? m : cap;
    if (k > 0) {
        std::vector<double> cum((size_t)k);
        ASX_CUDA(r, cudaMemcpy(cum.data(), r->samples, sizeof(double) * k, cudaMemcpyDeviceToHost));
        double prev = 0.0;
        for (int i = 0; i < k; i++) {
            q[i] = (cum[i] - prev) / sdt;
            prev = cum[i];
        }
    }
    return ASX_OK;
}

asx_status asx_get_clock(asx_raster *r, int scenario, double *t, double *dt, long long *step)
{
    if (!r) return ASX_EINVAL;
    if (scenario != 0) return fail(r, ASX_EINVAL, "scenario must be 0 for a single raster");
    asx_status st = set_device(r);
    if (st) return st;
    DevCtl *h;
    st = read_head(r, &h);
    if (st) return st;
    if (t) *t = h->t;
    if (dt) *dt = h->active ? h->dt : 0.0;
    if (step) *step = h->step;
    return ASX_OK;
}

}  // extern "C"
