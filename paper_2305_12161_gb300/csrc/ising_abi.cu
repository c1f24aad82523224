// C ABI of the library (declared in include/ising.h): context lifecycle, argument
// checks, error handling and dispatch to the kernels.  No kernel math lives here.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "../../include/ising.h"
#include "common.cuh"
#include "kernels.h"
#include <cufft.h>

using namespace ising;

struct ising_ctx {
    int L = 0, R = 0;
    uint64_t seed = 0;
    ising_opts opts{};
    Geom g{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t *lat = nullptr;     // packed store (PACKED form), or measurement copy (PLAIN form)
    uint32_t *lat_alt = nullptr; // second packed store of the fused sweep (VARIANT_ZFUSE)
    uint32_t *stage = nullptr;   // staging of ising_set_packed(ISING_PTR_HOST_ASYNC), one replica
    cudaStream_t copy_stream = nullptr;  // its host-to-device copies
    cudaEvent_t staged = nullptr;        // the staged words have landed (copy stream)
    cudaEvent_t stage_free = nullptr;    // the context stream has consumed them
    int8_t *plain = nullptr;     // PLAIN form lattice
    int64_t *rec_dev = nullptr;  // R records
    double *der_dev = nullptr;   // R x 4
    uint32_t *xt = nullptr;      // tensor-core correlation: bit-transposed lattice (lazy)
    int *dev_err = nullptr;      // set by a device-side bounded wait that gave up
    int xt_refused = 0;          // the tensor-core scratch could not be allocated (AUTO falls back)
    double wait_timeout_s = 2.0; // bound of each device-side wait (tensor-core path)
    int inject_stall = 0;        // test hook: the next tensor-core measurement loses one load
    int64_t t = 0;
    int poisoned = 0;
    int64_t launches = 0;
    SweepConfig cfg{};
    DcbGeom dcb{};  // double-checkerboard blocks (scheme DOUBLE)
    RadialPlans *radial = nullptr;  // cuFFT plans of the radial measurement (first use)
    char err[256] = {0};
};

namespace {

int fail(ising_ctx *c, int status, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
        if (status == ISING_ECUDA || status == ISING_ETIMEOUT) c->poisoned = status;
    }
    return status;
}

int cuda_fail(ising_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, ISING_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(ctx, call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);      \
    } while (0)

int check_ctx(ising_ctx *c)
{
    if (!c) return ISING_EINVAL;
    if (c->poisoned) return ISING_EPOISONED;
    return ISING_OK;
}

bool packed_L_ok(int L) { return (L >= 64 && L % 64 == 0) || L == 4 || L == 8 || L == 16 || L == 32; }

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t lattice_bytes_packed(int L, int R) { return (size_t)R * 2 * (size_t)make_geom(L).nw * sizeof(uint32_t); }

}  // namespace

namespace ising {

// Kernel configuration of the packed sweep from the variant, tile and depth options
// (variant 0: the default for L and R); false when it is not valid for L.
bool resolve_sweep_config(int L, int R, int variant, int tile_y, int tile_z, int depth, SweepConfig *out)
{
    SweepConfig cfg{};
    if (variant == 0) {
        cfg = default_sweep_config(L, R);
    } else {
        cfg = SweepConfig{variant, tile_y, tile_z, variant == VARIANT_ZFUSE ? depth : (depth ? depth : 3)};
        if ((cfg.variant == VARIANT_ZMARCH || cfg.variant == VARIANT_ZFAST || cfg.variant == VARIANT_ZDEEP ||
             cfg.variant == VARIANT_ZFUSE) &&
            (tile_y == 0 || tile_z == 0)) {
            if (L >= 256 && L % 256 == 0) {
                const int W4 = L / 256;
                if (!cfg.tile_y) cfg.tile_y = std::max(1, 256 / W4);
                if (!cfg.tile_z) cfg.tile_z = std::min(L, 16);
            }
        }
        if ((cfg.variant == VARIANT_ZFAST || cfg.variant == VARIANT_ZDEEP || cfg.variant == VARIANT_ZFUSE) &&
            L >= 256 && L % 256 == 0)
            cfg.tile_y = 256 / (L / 256);
        if (!sweep_config_valid(L, cfg)) return false;
    }
    *out = cfg;
    return true;
}

}  // namespace ising

extern "C" {

void ising_default_opts(ising_opts *o)
{
    if (!o) return;
    o->tie = ISING_TIE_GLAUBER;
    o->form = ISING_FORM_PACKED;
    o->stream = nullptr;
    o->device = -1;
    o->variant = 0;
    o->tile_y = 0;
    o->tile_z = 0;
    o->depth = 0;
    o->cycle = 0;
    o->corr = 0;
    o->scheme = ISING_SCHEME_CHECKERBOARD;
    o->block_x = 0;
    o->block_y = 0;
    o->block_z = 0;
    o->pdl = 1;
}

int64_t ising_record_len(int L)
{
    if (L < 4 || L % 2 != 0) return -1;
    return 3 + 3 * (int64_t)(L / 2 + 1);
}

int64_t ising_packed_words(int L)
{
    if (!packed_L_ok(L)) return -1;
    return 2 * make_geom(L).nw;
}

const char *ising_strerror(int s)
{
    switch (s) {
    case ISING_OK: return "ok";
    case ISING_EINVAL: return "invalid argument";
    case ISING_ENOMEM: return "out of memory";
    case ISING_ECUDA: return "CUDA error";
    case ISING_ETIMEOUT: return "device-side wait timed out";
    case ISING_EBUSY: return "busy";
    case ISING_EPOISONED: return "context poisoned by an earlier error";
    default: return "unknown status";
    }
}

const char *ising_last_error(const ising_ctx *c) { return c ? c->err : "null context"; }

int64_t ising_launch_count(const ising_ctx *c) { return c ? c->launches : -1; }

int ising_variants(int *ids, int cap)
{
    const int all[5] = {VARIANT_WORD, VARIANT_ZMARCH, VARIANT_ZFAST, VARIANT_ZDEEP, VARIANT_ZFUSE};
    if (!ids) return 5;
    int n = 0;
    for (int i = 0; i < 5 && n < cap; ++i) ids[n++] = all[i];
    return n;
}

int ising_destroy(ising_ctx *c)
{
    if (!c) return ISING_OK;
    {
        DeviceGuard dg(c->device);
        // stream-ordered frees: releasing a context does not synchronise other streams
        if (c->stream) {
            if (c->lat) cudaFreeAsync(c->lat, c->stream);
            if (c->lat_alt) cudaFreeAsync(c->lat_alt, c->stream);
            if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
            if (c->stage) cudaFreeAsync(c->stage, c->stream);
            if (c->plain) cudaFreeAsync(c->plain, c->stream);
            if (c->rec_dev) cudaFreeAsync(c->rec_dev, c->stream);
            if (c->der_dev) cudaFreeAsync(c->der_dev, c->stream);
            if (c->dev_err) cudaFreeAsync(c->dev_err, c->stream);
            if (c->xt) cudaFreeAsync(c->xt, c->stream);
            radial_plans_destroy(c->radial, c->stream);
            c->radial = nullptr;
            cudaStreamSynchronize(c->stream);
        }
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
        if (c->staged) cudaEventDestroy(c->staged);
        if (c->stage_free) cudaEventDestroy(c->stage_free);
    }
    delete c;
    return ISING_OK;
}

}  // extern "C"

namespace {

// Argument checks of a context and its sweep kernel choice (host arithmetic only: a bad
// configuration is refused before the device is touched).
int resolve_opts(int L, int R, const ising_opts &o, SweepConfig *cfg_out, DcbGeom *dcb_out)
{
    if (L < 4 || L % 2 != 0 || R < 1 || R > 65535) return ISING_EINVAL;
    if (o.tie < 0 || o.tie > 2 || (o.form != ISING_FORM_PACKED && o.form != ISING_FORM_PLAIN)) return ISING_EINVAL;
    if (o.cycle != ISING_CYCLE_01 && o.cycle != ISING_CYCLE_MIXED) return ISING_EINVAL;
    if (o.corr < ISING_CORR_AUTO || o.corr > ISING_CORR_TENSOR) return ISING_EINVAL;
    if (o.corr == ISING_CORR_TENSOR && !corr_mma_supported(L)) return ISING_EINVAL;
    // the measurement kernels always run on the packed store
    if (!packed_L_ok(L)) return ISING_EINVAL;
    if ((int64_t)L > 4096) return ISING_EINVAL;  // 32-bit Philox group index bound
    DcbGeom dcb{};
    if (o.scheme != ISING_SCHEME_CHECKERBOARD && o.scheme != ISING_SCHEME_DOUBLE) return ISING_EINVAL;
    if (o.scheme == ISING_SCHEME_DOUBLE &&
        (o.form != ISING_FORM_PACKED || !make_dcb_geom(L, o.block_x, o.block_y, o.block_z, &dcb)))
        return ISING_EINVAL;
    SweepConfig cfg{};
    if (!resolve_sweep_config(L, R, o.variant, o.tile_y, o.tile_z, o.depth, &cfg)) return ISING_EINVAL;
    if (o.pdl != 0 && o.pdl != 1) return ISING_EINVAL;
    cfg.pdl = o.pdl;
    if (cfg_out) *cfg_out = cfg;
    if (dcb_out) *dcb_out = dcb;
    return ISING_OK;
}

// Device memory of a context, by buffer.  ising_create_ex allocates exactly the first six
// at creation; the correlation scratch is allocated by the first measurement that runs the
// tensor-core path and then kept.
struct Footprint {
    size_t lat, lat_alt, plain, rec, der, err, corr;
    size_t total() const { return lat + lat_alt + plain + rec + der + err + corr; }
};

// Whether a measurement of this context runs the tensor-core correlation (before any
// allocation was refused).
bool wants_tensor_corr(int L, const ising_opts &o)
{
    return o.corr == ISING_CORR_TENSOR || (o.corr == ISING_CORR_AUTO && L >= 512 && corr_mma_supported(L));
}

Footprint footprint_of(int L, int R, const ising_opts &o, const SweepConfig &cfg)
{
    Footprint f{};
    f.lat = lattice_bytes_packed(L, R);
    f.lat_alt = (cfg.variant == VARIANT_ZFUSE && o.form == ISING_FORM_PACKED && o.scheme == ISING_SCHEME_CHECKERBOARD)
                    ? f.lat
                    : 0;
    f.plain = o.form == ISING_FORM_PLAIN ? (size_t)R * (size_t)L * L * L : 0;
    f.rec = sizeof(int64_t) * (size_t)R * (size_t)ising_record_len(L);
    f.der = sizeof(double) * 4 * (size_t)R;
    f.err = sizeof(int) * 4;
    f.corr = wants_tensor_corr(L, o) ? corr_mma_scratch_bytes(L, R) : 0;
    return f;
}

}  // namespace

extern "C" {

int64_t ising_footprint_bytes(int L, int R, const ising_opts *opts)
{
    ising_opts o;
    ising_default_opts(&o);
    if (opts) o = *opts;
    SweepConfig cfg{};
    if (resolve_opts(L, R, o, &cfg, nullptr) != ISING_OK) return -1;
    return (int64_t)footprint_of(L, R, o, cfg).total();
}

int ising_create_ex(ising_ctx **out, int L, int R, uint64_t seed, const ising_opts *opts)
{
    if (!out) return ISING_EINVAL;
    *out = nullptr;
    ising_opts o;
    ising_default_opts(&o);
    if (opts) o = *opts;
    SweepConfig cfg{};
    DcbGeom dcb{};
    const int st = resolve_opts(L, R, o, &cfg, &dcb);
    if (st != ISING_OK) return st;
    const Footprint fp = footprint_of(L, R, o, cfg);
    ising_ctx *c = new (std::nothrow) ising_ctx();
    if (!c) return ISING_ENOMEM;
    c->L = L;
    c->R = R;
    c->seed = seed;
    c->opts = o;
    c->g = make_geom(L);
    c->dcb = dcb;
    c->cfg = cfg;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete c;
        return ISING_ECUDA;
    }
    c->device = dev;
    DeviceGuard dg(dev);
    auto bail = [&](int s) {
        ising_destroy(c);
        return s;
    };
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(ISING_ECUDA);
        c->own_stream = true;
    }
    // stream-ordered allocations (no implicit device synchronisation); sizes from the same
    // accounting that ising_footprint_bytes reports
    const size_t pbytes = fp.lat;
    if (cudaMallocAsync((void **)&c->lat, fp.lat, c->stream) != cudaSuccess) return bail(ISING_ENOMEM);
    if (fp.lat_alt && cudaMallocAsync((void **)&c->lat_alt, fp.lat_alt, c->stream) != cudaSuccess)
        return bail(ISING_ENOMEM);
    if (fp.plain && cudaMallocAsync((void **)&c->plain, fp.plain, c->stream) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMallocAsync((void **)&c->rec_dev, fp.rec, c->stream) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMallocAsync((void **)&c->der_dev, fp.der, c->stream) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMallocAsync((void **)&c->dev_err, fp.err, c->stream) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMemsetAsync(c->dev_err, 0, fp.err, c->stream) != cudaSuccess) return bail(ISING_ECUDA);
    cudaError_t e;
    if (o.form == ISING_FORM_PLAIN) {
        e = launch_init_plain(c->plain, L, R, seed, c->stream);
    } else {
        // padded words (L < 64) must hold zeros beyond the row's L/2 bits
        if (L < 64) {
            e = cudaMemsetAsync(c->lat, 0, pbytes, c->stream);
            if (e != cudaSuccess) return bail(ISING_ECUDA);
        }
        e = launch_init_packed(c->lat, L, R, seed, c->stream);
    }
    c->launches += 1;
    if (e != cudaSuccess) return bail(ISING_ECUDA);
    *out = c;
    return ISING_OK;
}

int ising_create(ising_ctx **out, int L, int R, uint64_t seed) { return ising_create_ex(out, L, R, seed, nullptr); }

int ising_reinit(ising_ctx *c, uint64_t seed)
{
    int s = check_ctx(c);
    if (s) return s;
    DeviceGuard dg(c->device);
    c->seed = seed;
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, launch_init_plain(c->plain, c->L, c->R, seed, c->stream));
    } else {
        CK(c, launch_init_packed(c->lat, c->L, c->R, seed, c->stream));
    }
    c->launches += 1;
    c->t = 0;
    return ISING_OK;
}

int ising_init_menger(ising_ctx *c, int k)
{
    int s = check_ctx(c);
    if (s) return s;
    if (k < 0 || k > 8) return fail(c, ISING_EINVAL, "Menger iteration must be in 0..8");
    DeviceGuard dg(c->device);
    if (c->L < 64) CK(c, cudaMemsetAsync(c->lat, 0, lattice_bytes_packed(c->L, c->R), c->stream));
    CK(c, launch_init_menger(c->lat, c->L, c->R, c->seed, k, c->stream));
    c->launches += 1;
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, launch_unpack(c->lat, c->plain, c->L, c->R, c->stream));
        c->launches += 1;
    }
    c->t = 0;
    return ISING_OK;
}

int ising_sweep(ising_ctx *c, int64_t n)
{
    int s = check_ctx(c);
    if (s) return s;
    if (n < 0) return fail(c, ISING_EINVAL, "negative sweep count");
    if (c->t + n > (int64_t)0xffffffffll) return fail(c, ISING_EINVAL, "sweep counter beyond 2^32");
    if (n == 0) return ISING_OK;
    DeviceGuard dg(c->device);
    cudaError_t e;
    if (c->opts.scheme == ISING_SCHEME_DOUBLE)
        e = launch_sweeps_dcb(c->lat, c->L, c->R, c->seed, c->opts.tie, c->t, n, c->opts.cycle, c->dcb, c->stream,
                              &c->launches);
    else if (c->opts.form == ISING_FORM_PLAIN)
        e = launch_sweeps_plain(c->plain, c->L, c->R, c->seed, c->opts.tie, c->t, n, c->opts.cycle, c->stream,
                                &c->launches);
    else if (c->cfg.variant == VARIANT_ZFUSE)
        e = launch_sweeps_fused(&c->lat, &c->lat_alt, c->L, c->R, c->seed, c->opts.tie, c->t, n, c->opts.cycle,
                                c->cfg.tile_z, c->cfg.depth, c->dev_err, c->wait_timeout_s, c->stream, &c->launches,
                                c->cfg.pdl != 0);
    else
        e = launch_sweeps_packed(c->lat, c->L, c->R, c->seed, c->opts.tie, c->t, n, c->opts.cycle, c->cfg, c->stream,
                                 &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
    c->t += n;
    return ISING_OK;
}

// Synchronise the context's stream and report a device-side wait that gave up (the
// tensor-core correlation's bounded mbarrier waits) as ISING_ETIMEOUT, which poisons the
// context.
static int check_device_waits(ising_ctx *c)
{
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h == 4) return fail(c, ISING_ETIMEOUT, "fused sweep: a bounded wait for a copy gave up");
    if (h) return fail(c, ISING_ETIMEOUT, "tensor-core correlation: a bounded device-side wait gave up (code %d)", h);
    return ISING_OK;
}

int64_t ising_radial_bins(int L)
{
    if (L < 4 || L % 2 != 0 || L > 4096) return -1;
    return radial_nbins(L);
}

int ising_measure_radial(ising_ctx *c, int replica, int precision, double cval, double *C, double *S, int64_t *count,
                         double *ell, int64_t *inexact)
{
    int s = check_ctx(c);
    if (s) return s;
    if (replica < 0 || replica >= c->R) return fail(c, ISING_EINVAL, "replica out of range");
    if (precision != ISING_FFT_SINGLE && precision != ISING_FFT_DOUBLE) return fail(c, ISING_EINVAL, "precision");
    if (!C || !S) return fail(c, ISING_EINVAL, "null output");
    DeviceGuard dg(c->device);
    if (!c->radial && !(c->radial = radial_plans_create())) return fail(c, ISING_ENOMEM, "radial plans");
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, launch_pack(c->plain, c->lat, c->L, c->R, c->stream));
        c->launches += 1;
    }
    const int64_t nb = radial_nbins(c->L);
    double *out = nullptr;
    int64_t *cnt = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(double) * (size_t)(2 * nb + 1), c->stream) != cudaSuccess)
        return fail(c, ISING_ENOMEM, "radial output");
    if (cudaMallocAsync((void **)&cnt, sizeof(int64_t) * (size_t)(nb + 1), c->stream) != cudaSuccess) {
        cudaFreeAsync(out, c->stream);
        return fail(c, ISING_ENOMEM, "radial output");
    }
    int cs = 0;
    const uint32_t *lat_r = c->lat + 2 * (int64_t)replica * c->g.nw;
    cudaError_t e = launch_radial(c->radial, lat_r, c->L, precision, cval, out, cnt, c->stream, &c->launches, &cs);
    if (e != cudaSuccess) {
        cudaFreeAsync(cnt, c->stream);
        cudaFreeAsync(out, c->stream);
        if (e == cudaErrorMemoryAllocation || cs == CUFFT_ALLOC_FAILED) {
            cudaGetLastError();  // a failed allocation is not sticky
            return fail(c, ISING_ENOMEM, "radial measurement: scratch of %zu bytes",
                        radial_scratch_bytes(c->L, precision));
        }
        if (cs) return fail(c, ISING_ECUDA, "cuFFT status %d", cs);
        return cuda_fail(c, e, "radial measurement");
    }
    std::vector<double> h(2 * nb + 1);
    std::vector<int64_t> hc(nb + 1);
    CK(c, cudaMemcpyAsync(h.data(), out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(hc.data(), cnt, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, c->stream));
    cudaFreeAsync(cnt, c->stream);
    cudaFreeAsync(out, c->stream);
    CK(c, cudaStreamSynchronize(c->stream));
    std::copy(h.begin(), h.begin() + nb, C);
    std::copy(h.begin() + nb, h.begin() + 2 * nb, S);
    if (ell) *ell = h[2 * nb];
    if (count) std::copy(hc.begin(), hc.begin() + nb, count);
    if (inexact) *inexact = hc[nb];
    return ISING_OK;
}

int ising_release_scratch(ising_ctx *c)
{
    int s = check_ctx(c);
    if (s) return s;
    DeviceGuard dg(c->device);
    radial_release(c->radial, c->stream);
    if (c->xt) cudaFreeAsync(c->xt, c->stream);
    c->xt = nullptr;
    if (c->stage) {  // the copy stream has finished with it before the context stream frees it
        CK(c, cudaStreamSynchronize(c->copy_stream));
        cudaFreeAsync(c->stage, c->stream);
        c->stage = nullptr;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return ISING_OK;
}

int ising_inject_corr_stall(ising_ctx *c, double timeout_s)
{
    int s = check_ctx(c);
    if (s) return s;
    if (!(timeout_s > 0) || timeout_s > 60) return fail(c, ISING_EINVAL, "timeout must be in (0, 60] s");
    c->wait_timeout_s = timeout_s;
    c->inject_stall = 1;
    return ISING_OK;
}

int ising_measure_ex(ising_ctx *c, int64_t *rec, double *derived, double cval, unsigned flags)
{
    int s = check_ctx(c);
    if (s) return s;
    if (flags & ~(ISING_MEAS_DEVICE | ISING_MEAS_CONNECTED | ISING_MEAS_NO_CORR))
        return fail(c, ISING_EINVAL, "unknown measure flags");
    DeviceGuard dg(c->device);
    const bool dev = flags & ISING_MEAS_DEVICE;
    const bool corr = !(flags & ISING_MEAS_NO_CORR);
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, launch_pack(c->plain, c->lat, c->L, c->R, c->stream));
        c->launches += 1;
    }
    int64_t *rdst = (dev && rec) ? rec : c->rec_dev;
    int method = CORR_NONE;
    if (corr) {
        method = CORR_POPCOUNT;
        if (wants_tensor_corr(c->L, c->opts) && !(c->opts.corr == ISING_CORR_AUTO && c->xt_refused))
            method = CORR_TENSOR;
    }
    if (method == CORR_TENSOR && !c->xt) {
        const size_t bytes = corr_mma_scratch_bytes(c->L, c->R);
        if (cudaMallocAsync((void **)&c->xt, bytes, c->stream) != cudaSuccess) {
            c->xt = nullptr;
            cudaGetLastError();  // a failed allocation is not sticky
            if (c->opts.corr == ISING_CORR_TENSOR) return fail(c, ISING_ENOMEM, "correlation scratch");
            c->xt_refused = 1;   // automatic choice: the bit-count path needs no scratch
            method = CORR_POPCOUNT;
        }
    }
    const int inject = method == CORR_TENSOR ? c->inject_stall : 0;
    c->inject_stall = 0;
    CK(c, launch_measure(c->lat, c->L, c->R, c->t, method, rdst, c->stream, &c->launches, c->xt, c->dev_err,
                         c->wait_timeout_s, inject));
    double *ddst = nullptr;
    if (derived) {
        ddst = dev ? derived : c->der_dev;
        CK(c, launch_derived(rdst, c->L, c->R, cval, flags & ISING_MEAS_CONNECTED, ddst, c->stream, &c->launches));
    }
    if (!dev) {
        const int64_t RL = ising_record_len(c->L);
        if (rec) CK(c, cudaMemcpyAsync(rec, rdst, sizeof(int64_t) * RL * c->R, cudaMemcpyDeviceToHost, c->stream));
        if (derived)
            CK(c, cudaMemcpyAsync(derived, ddst, sizeof(double) * 4 * c->R, cudaMemcpyDeviceToHost, c->stream));
        return check_device_waits(c);
    }
    return ISING_OK;
}

int ising_measure(ising_ctx *c, int64_t *out)
{
    if (!out) return c ? fail(c, ISING_EINVAL, "null output") : ISING_EINVAL;
    return ising_measure_ex(c, out, nullptr, 0.5, 0u);
}

int ising_get_spins(ising_ctx *c, int replica, int8_t *host_out)
{
    int s = check_ctx(c);
    if (s) return s;
    if (!host_out || replica < 0 || replica >= c->R) return fail(c, ISING_EINVAL, "bad replica or buffer");
    DeviceGuard dg(c->device);
    const size_t N = (size_t)c->L * c->L * c->L;
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, cudaMemcpyAsync(host_out, c->plain + (size_t)replica * N, N, cudaMemcpyDeviceToHost, c->stream));
    } else {
        int8_t *tmp = nullptr;
        if (cudaMallocAsync(&tmp, N, c->stream) != cudaSuccess) return fail(c, ISING_ENOMEM, "staging buffer");
        cudaError_t e = launch_unpack(c->lat + (size_t)replica * 2 * c->g.nw, tmp, c->L, 1, c->stream);
        c->launches += 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, N, cudaMemcpyDeviceToHost, c->stream);
        cudaFreeAsync(tmp, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_spins");
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return ISING_OK;
}

int ising_set_spins(ising_ctx *c, int replica, const int8_t *host_in)
{
    int s = check_ctx(c);
    if (s) return s;
    if (!host_in || replica < 0 || replica >= c->R) return fail(c, ISING_EINVAL, "bad replica or buffer");
    const size_t N = (size_t)c->L * c->L * c->L;
    for (size_t i = 0; i < N; ++i)
        if (host_in[i] != 1 && host_in[i] != -1) return fail(c, ISING_EINVAL, "spin values must be +1 or -1");
    DeviceGuard dg(c->device);
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, cudaMemcpyAsync(c->plain + (size_t)replica * N, host_in, N, cudaMemcpyHostToDevice, c->stream));
    } else {
        int8_t *tmp = nullptr;
        if (cudaMallocAsync(&tmp, N, c->stream) != cudaSuccess) return fail(c, ISING_ENOMEM, "staging buffer");
        cudaError_t e = cudaMemcpyAsync(tmp, host_in, N, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_pack(tmp, c->lat + (size_t)replica * 2 * c->g.nw, c->L, 1, c->stream);
        c->launches += 1;
        cudaFreeAsync(tmp, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_spins");
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return ISING_OK;
}

int ising_get_packed(ising_ctx *c, int replica, uint32_t *words, unsigned flags)
{
    int s = check_ctx(c);
    if (s) return s;
    if (!words || replica < 0 || replica >= c->R || (flags & ~ISING_PTR_DEVICE))
        return fail(c, ISING_EINVAL, "bad replica, buffer or flags");
    DeviceGuard dg(c->device);
    if (c->opts.form == ISING_FORM_PLAIN) {
        CK(c, launch_pack(c->plain, c->lat, c->L, c->R, c->stream));
        c->launches += 1;
    }
    const size_t bytes = 2 * (size_t)c->g.nw * sizeof(uint32_t);
    const bool dev = flags & ISING_PTR_DEVICE;
    CK(c, cudaMemcpyAsync(words, c->lat + (size_t)replica * 2 * c->g.nw, bytes,
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!dev) CK(c, cudaStreamSynchronize(c->stream));
    return ISING_OK;
}

int ising_set_packed(ising_ctx *c, int replica, const uint32_t *words, unsigned flags)
{
    int s = check_ctx(c);
    if (s) return s;
    if (!words || replica < 0 || replica >= c->R || (flags & ~(ISING_PTR_DEVICE | ISING_PTR_HOST_ASYNC)) ||
        flags == (ISING_PTR_DEVICE | ISING_PTR_HOST_ASYNC))
        return fail(c, ISING_EINVAL, "bad replica, buffer or flags");
    const bool dev = flags & ISING_PTR_DEVICE, host_async = flags & ISING_PTR_HOST_ASYNC;
    if (!dev && c->L < 64) {
        const uint32_t m = row_mask(c->g.RB);
        for (int64_t i = 0; i < 2 * c->g.nw; ++i)
            if (words[i] & ~m) return fail(c, ISING_EINVAL, "padding bits must be zero");
    }
    DeviceGuard dg(c->device);
    const size_t bytes = 2 * (size_t)c->g.nw * sizeof(uint32_t);
    if (host_async) {
        if (!c->stage) {
            if (cudaMallocAsync((void **)&c->stage, bytes, c->stream) != cudaSuccess) {
                cudaGetLastError();
                c->stage = nullptr;
                return fail(c, ISING_ENOMEM, "staging buffer of %zu bytes", bytes);
            }
            if (!c->copy_stream) CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
            if (!c->staged) CK(c, cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming));
            if (!c->stage_free) CK(c, cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming));
            CK(c, cudaEventRecord(c->stage_free, c->stream));  // the allocation is stream-ordered
        }
        // the copy stream waits only for the previous staged words to be consumed, not for
        // the work queued on the context's stream
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->stage_free, 0));
        CK(c, cudaMemcpyAsync(c->stage, words, bytes, cudaMemcpyHostToDevice, c->copy_stream));
        CK(c, cudaEventRecord(c->staged, c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->staged, 0));
        CK(c, cudaMemcpyAsync(c->lat + (size_t)replica * 2 * c->g.nw, c->stage, bytes, cudaMemcpyDeviceToDevice,
                              c->stream));
        CK(c, cudaEventRecord(c->stage_free, c->stream));
    } else {
        CK(c, cudaMemcpyAsync(c->lat + (size_t)replica * 2 * c->g.nw, words, bytes,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    }
    if (c->opts.form == ISING_FORM_PLAIN) {
        // expand only this replica into the byte lattice
        const size_t N = (size_t)c->L * c->L * c->L;
        CK(c, launch_unpack(c->lat + (size_t)replica * 2 * c->g.nw, c->plain + (size_t)replica * N, c->L, 1,
                            c->stream));
        c->launches += 1;
    }
    if (!dev && !host_async) CK(c, cudaStreamSynchronize(c->stream));
    return ISING_OK;
}

int ising_get_time(ising_ctx *c, int64_t *t)
{
    if (!c || !t) return ISING_EINVAL;
    *t = c->t;
    return ISING_OK;
}

int ising_set_time(ising_ctx *c, int64_t t)
{
    int s = check_ctx(c);
    if (s) return s;
    if (t < 0 || t > (int64_t)0xffffffffll) return fail(c, ISING_EINVAL, "time out of range");
    c->t = t;
    return ISING_OK;
}

int ising_sync(ising_ctx *c)
{
    int s = check_ctx(c);
    if (s) return s;
    DeviceGuard dg(c->device);
    return check_device_waits(c);
}

int ising_tune_sweep(int L, int replicas, int probe_mcs, const ising_opts *base, ising_opts *best,
                     double *best_ms_per_mcs)
{
    if (!best || probe_mcs < 1 || replicas < 1 || !packed_L_ok(L)) return ISING_EINVAL;
    ising_opts o;
    ising_default_opts(&o);
    if (base) o = *base;
    if (o.form != ISING_FORM_PACKED || o.scheme != ISING_SCHEME_CHECKERBOARD) return ISING_EINVAL;
    std::vector<SweepConfig> cands;
    cands.push_back(SweepConfig{VARIANT_WORD, 0, 0, 0});
    const int tzs[] = {4, 8, 16, 32, 64};
    if (L >= 256 && L % 256 == 0) {
        const int W4 = L / 256;
        for (int ty = 1; ty <= L; ty *= 2)
            for (int tz : tzs) {
                const SweepConfig c{VARIANT_ZMARCH, ty, tz, 0};
                if (ty * W4 >= 64 && sweep_config_valid(L, c)) cands.push_back(c);
            }
        for (int tz : tzs) {
            const SweepConfig c{VARIANT_ZFAST, 256 / W4, tz, 0};
            if (sweep_config_valid(L, c)) cands.push_back(c);
            for (int d = 2; d <= 4; ++d) {
                const SweepConfig cd{VARIANT_ZDEEP, 256 / W4, tz, d};
                if (sweep_config_valid(L, cd)) cands.push_back(cd);
            }
        }
        // thin z-blocks (4, 8 planes) give small lattices enough tiles to fill the GPU
        for (int tz : {4, 8, 16, 32, 64, 128})
            for (int mb : {1, 2, 3, 9, 10, 11, 18, 19, 25, 26, 27}) {
                if (tz < 16 && L > 512) continue;
                const SweepConfig cf{VARIANT_ZFUSE, 256 / W4, tz, mb};
                if (sweep_config_valid(L, cf)) cands.push_back(cf);
            }
    }
    // The fused sweep holds a second packed store, so it is kept only when it beats the best
    // single-store kernel by more than the run-to-run spread of these probes (3%).
    double best_ms = 1e300, best_single_ms = 1e300, best_fused_ms = 1e300;
    ising_opts best_single{}, best_fused{};
    bool found = false;
    for (const SweepConfig &c : cands) {
        ising_opts oc = o;
        oc.variant = c.variant;
        oc.tile_y = c.tile_y;
        oc.tile_z = c.tile_z;
        oc.depth = c.depth;
        ising_ctx *ctx = nullptr;
        int st = ising_create_ex(&ctx, L, replicas, 1, &oc);
        if (st != ISING_OK) continue;
        cudaEvent_t a = nullptr, b = nullptr;
        float ms = 0.f;
        bool ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
        ok = ok && ising_sweep(ctx, 2) == ISING_OK;
        ok = ok && cudaEventRecord(a, ctx->stream) == cudaSuccess;
        ok = ok && ising_sweep(ctx, probe_mcs) == ISING_OK;
        ok = ok && cudaEventRecord(b, ctx->stream) == cudaSuccess;
        ok = ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        ising_destroy(ctx);
        if (!ok) return ISING_ECUDA;
        const double per = ms / probe_mcs;
        if (c.variant == VARIANT_ZFUSE) {
            if (per < best_fused_ms) best_fused_ms = per, best_fused = oc;
        } else if (per < best_single_ms) {
            best_single_ms = per, best_single = oc;
        }
        found = true;
    }
    if (!found) return ISING_EINVAL;
    if (best_fused_ms < best_single_ms / 1.03) {
        best_ms = best_fused_ms;
        *best = best_fused;
    } else {
        best_ms = best_single_ms;
        *best = best_single;
    }
    if (best_ms_per_mcs) *best_ms_per_mcs = best_ms;
    return ISING_OK;
}

}  // extern "C"
