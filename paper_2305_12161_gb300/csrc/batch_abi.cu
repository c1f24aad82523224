// C ABI of the batched form (declared in include/ising.h): a batch of lattice classes
// (L, replicas, seed) advanced together by one persistent cooperative launch per run
// segment, with the larger classes streamed beside it by single-lattice sweep kernels on
// side streams, measured per class (one class per stream) with the single-lattice
// measurement kernels, and a whole log-spaced schedule (segments + measurements) captured
// into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "batch.h"
#include "common.cuh"
#include "kernels.h"

using namespace ising;

namespace {

struct BatchClass {
    int L, R;
    uint64_t seed;
    uint32_t *lat;       // R * 2 * nw words
    int64_t rec_off;     // offset of this class's records in a batch record block
    int64_t der_off;     // offset (in replicas) of this class's derived rows
    int streamed;        // swept by a single-lattice sweep kernel instead of the persistent one
    SweepConfig cfg;     // that kernel's configuration (streamed classes)
    uint32_t *alt;       // second store of the fused whole-sweep kernel (allocated when chosen)
    uint32_t *xt;        // tensor-core correlation scratch (L >= 512), else null: bit counts
};

bool packed_L_ok(int L) { return (L >= 64 && L % 64 == 0) || L == 4 || L == 8 || L == 16 || L == 32; }

}  // namespace

struct ising_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // streamed classes run on side streams forked from and joined back into `stream` within
    // each segment (ev[0]: fork, ev[1 + i]: join of side[i]); with `overlap` every streamed
    // class has a side stream and runs beside the persistent launch, otherwise the first
    // one runs on `stream` after it.  Measurements fork one class per stream the same way.
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    int overlap = 0;
    int rule = 0;
    std::vector<BatchClass> cls;
    int64_t nlat = 0, rec_words = 0;
    int64_t t = 0;
    int poisoned = 0;
    int64_t launches = 0;
    char err[256] = {0};
    // plan
    std::vector<BatchLattice> h_lats;
    std::vector<BatchTask> h_tasks;
    BatchLattice *d_lats = nullptr;
    BatchTask *d_tasks = nullptr;
    unsigned *d_barriers = nullptr;
    int ngroups = 0;
    int *d_status = nullptr;
    unsigned long long *d_cta_ns = nullptr;
    int smem = 0, occ = 0, sms = 0, capacity = 0;
    double w_local = 1.0, w_group = 1.0;
    uint64_t timeout_ns = 2000000000ull;
    int missing_cta = -1;
    int stream_min_L = 256;  // classes with L >= this (and L % 256 == 0) are streamed
    // measurement scratch
    int64_t *d_rec = nullptr;
    double *d_der = nullptr;
    // cached schedule graph
    cudaGraphExec_t gexec = nullptr;
    std::vector<int64_t> gkey;
};

namespace {

int bfail(ising_batch *b, int status, const char *msg)
{
    if (b) {
        snprintf(b->err, sizeof(b->err), "%s", msg);
        if (status == ISING_ECUDA || status == ISING_ETIMEOUT) b->poisoned = status;
    }
    return status;
}

int bcuda(ising_batch *b, cudaError_t e, const char *where)
{
    char m[200];
    snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
    return bfail(b, ISING_ECUDA, m);
}

#define BCK(b, call)                                                \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call);        \
    } while (0)

int bcheck(ising_batch *b)
{
    if (!b) return ISING_EINVAL;
    if (b->poisoned) return ISING_EPOISONED;
    return ISING_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard()
    {
        int c = -1;
        if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev);
    }
};

int64_t lattice_bytes(int L) { return 2 * make_geom(L).nw * 4; }

// Build the CTA work list: LOCAL tasks pack consecutive small lattices, GROUP tasks
// split a large lattice into slabs; sizes follow expected cost (spins x mode weight),
// scaled until the whole list is co-resident (<= capacity CTAs).
int build_plan(ising_batch *b)
{
    std::vector<BatchTask> tasks;
    const int cap = b->capacity;
    double total = 0;
    for (const auto &l : b->h_lats) {
        const double N = (double)l.L * l.L * l.L;
        total += N * (lattice_bytes(l.L) <= b->smem ? b->w_local : b->w_group);
    }
    double T = total / cap;
    for (int iter = 0; iter < 200; ++iter) {
        tasks.clear();
        int group = 0;
        int i = 0;
        const int n = (int)b->h_lats.size();
        while (i < n) {
            const BatchLattice &l = b->h_lats[i];
            const double N = (double)l.L * l.L * l.L;
            if (lattice_bytes(l.L) <= b->smem) {
                // pack consecutive small lattices until the task reaches T
                int j = i;
                double c = 0;
                while (j < n && lattice_bytes(b->h_lats[j].L) <= b->smem) {
                    const double Nj = (double)b->h_lats[j].L * b->h_lats[j].L * b->h_lats[j].L;
                    if (j > i && c + 0.5 * Nj * b->w_local > T) break;
                    c += Nj * b->w_local;
                    ++j;
                }
                tasks.push_back(BatchTask{BATCH_LOCAL, i, j - i, 0, 0, 1});
                i = j;
            } else {
                const Geom g = make_geom(l.L);
                const int64_t units = g.L >= 64 ? g.nw / 4 : g.nw;
                int size = (int)std::llround(N * b->w_group / T);
                size = std::max(1, std::min<int>(size, (int)std::min<int64_t>(units, cap)));
                for (int r = 0; r < size; ++r) tasks.push_back(BatchTask{BATCH_GROUP, i, 1, group, r, size});
                ++group;
                ++i;
            }
        }
        if ((int)tasks.size() <= cap) {
            b->ngroups = group;
            b->h_tasks = tasks;
            return ISING_OK;
        }
        T *= 1.05;
    }
    return ISING_EINVAL;
}

int upload_plan(ising_batch *b)
{
    cudaFree(b->d_tasks);
    cudaFree(b->d_barriers);
    cudaFree(b->d_cta_ns);
    b->d_tasks = nullptr;
    b->d_barriers = nullptr;
    b->d_cta_ns = nullptr;
    const size_t nt = b->h_tasks.size();
    if (cudaMalloc(&b->d_tasks, std::max<size_t>(1, nt) * sizeof(BatchTask)) != cudaSuccess) return ISING_ENOMEM;
    if (cudaMalloc(&b->d_barriers, sizeof(unsigned) * (size_t)std::max(1, b->ngroups)) != cudaSuccess)
        return ISING_ENOMEM;
    if (cudaMalloc(&b->d_cta_ns, std::max<size_t>(1, nt) * sizeof(unsigned long long)) != cudaSuccess)
        return ISING_ENOMEM;
    if (nt)
        BCK(b, cudaMemcpyAsync(b->d_tasks, b->h_tasks.data(), nt * sizeof(BatchTask), cudaMemcpyHostToDevice,
                               b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->gkey.clear();
    }
    return ISING_OK;
}

// Enqueue one segment of n MCS (split at 2^30 sweeps per launch).
int enqueue_segment(ising_batch *b, int64_t n, unsigned long long *cta_ns)
{
    while (n > 0) {
        const int chunk = (int)std::min<int64_t>(n, 1 << 30);
        int nstreamed = 0, si = 0;
        for (const auto &k : b->cls) nstreamed += k.streamed;
        const bool persistent = !b->h_tasks.empty();
        // side streams: every streamed class when they overlap the persistent launch, else all
        // but the first, which follows the persistent launch on the batch's stream
        const int first_side = (b->overlap && persistent) ? 0 : 1;
        // fork before the persistent launch when the streamed classes overlap it, after it
        // otherwise
        if (first_side == 0 && nstreamed > 0) BCK(b, cudaEventRecord(b->ev[0], b->stream));
        if (persistent) {
            BCK(b, cudaMemsetAsync(b->d_barriers, 0, sizeof(unsigned) * (size_t)std::max(1, b->ngroups), b->stream));
            BCK(b, launch_batch(b->d_tasks, (int)b->h_tasks.size(), b->d_lats, b->rule, (uint32_t)b->t, chunk,
                                b->d_barriers, b->d_status, b->timeout_ns, b->missing_cta, cta_ns, b->smem,
                                b->stream));
            b->launches += 1;
        }
        if (first_side == 1 && nstreamed > 1) BCK(b, cudaEventRecord(b->ev[0], b->stream));
        // the streamed classes, each on its own stream: their short launches (a few
        // microseconds of work each) overlap instead of waiting for one another
        for (const auto &k : b->cls) {
            if (!k.streamed) continue;
            const int sj = si + (1 - first_side);  // side stream index + 1 (0: the batch's stream)
            cudaStream_t st = b->stream;
            if (sj > 0) {
                st = b->side[sj - 1];
                BCK(b, cudaStreamWaitEvent(st, b->ev[0], 0));
            }
            if (k.cfg.variant == VARIANT_ZFUSE) {
                // whole sweeps between the two stores: an even count ends in k.lat again, and
                // an odd last sweep runs in place, so a segment always leaves the state there
                const int even = chunk & ~1;
                uint32_t *cur = k.lat, *nxt = k.alt;
                if (even)
                    BCK(b, launch_sweeps_fused(&cur, &nxt, k.L, k.R, k.seed, b->rule, b->t, even, 0, k.cfg.tile_z,
                                               k.cfg.depth, b->d_status, (double)b->timeout_ns * 1e-9, st,
                                               &b->launches, k.cfg.pdl != 0));
                if (chunk & 1)
                    BCK(b, launch_sweeps_packed(k.lat, k.L, k.R, k.seed, b->rule, b->t + even, 1, 0,
                                                default_sweep_config(k.L, k.R), st, &b->launches));
            } else {
                BCK(b, launch_sweeps_packed(k.lat, k.L, k.R, k.seed, b->rule, b->t, chunk, 0, k.cfg, st,
                                            &b->launches));
            }
            if (sj > 0) BCK(b, cudaEventRecord(b->ev[sj], st));
            ++si;
        }
        for (int j = 1; j <= si - first_side; ++j) BCK(b, cudaStreamWaitEvent(b->stream, b->ev[j], 0));
        b->t += chunk;
        n -= chunk;
    }
    return ISING_OK;
}

int enqueue_measure(ising_batch *b, int64_t *rec, double *der, double c, unsigned flags)
{
    // one class per stream (class 0 on the batch's stream, class i on side stream i - 1): the
    // classes write disjoint parts of rec and der and share no scratch
    const bool corr = !(flags & ISING_MEAS_NO_CORR);
    const int nc = (int)b->cls.size();
    if (nc > 1) BCK(b, cudaEventRecord(b->ev[0], b->stream));
    for (int i = 0; i < nc; ++i) {
        const auto &k = b->cls[i];
        cudaStream_t st = i == 0 ? b->stream : b->side[i - 1];
        if (i > 0) BCK(b, cudaStreamWaitEvent(st, b->ev[0], 0));
        const int method = !corr ? CORR_NONE : (k.xt ? CORR_TENSOR : CORR_POPCOUNT);
        BCK(b, launch_measure(k.lat, k.L, k.R, b->t, method, rec + k.rec_off, st, &b->launches, k.xt, b->d_status,
                              (double)b->timeout_ns * 1e-9));
        if (der)
            BCK(b, launch_derived(rec + k.rec_off, k.L, k.R, c, flags & ISING_MEAS_CONNECTED, der + 4 * k.der_off,
                                  st, &b->launches));
        if (i > 0) BCK(b, cudaEventRecord(b->ev[i], st));
    }
    for (int i = 1; i < nc; ++i) BCK(b, cudaStreamWaitEvent(b->stream, b->ev[i], 0));
    return ISING_OK;
}

int read_status(ising_batch *b)
{
    int st = 0;
    BCK(b, cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    // status codes: 1 a group barrier of the batch kernel (or the first wait of a tensor-core
    // correlation CTA) ran out, 2 and 3 later waits of the tensor-core correlation, 4 a copy
    // wait of the fused sweep
    if (st == BATCH_STATUS_TIMEOUT)
        return bfail(b, ISING_ETIMEOUT, "a group barrier of the batch kernel or a correlation wait timed out");
    if (st == 4) return bfail(b, ISING_ETIMEOUT, "fused sweep of a streamed class: a bounded wait for a copy gave up");
    if (st) return bfail(b, ISING_ETIMEOUT, "tensor-core correlation: a bounded device-side wait gave up");
    return ISING_OK;
}

// Split the classes between the persistent kernel and the single-lattice kernels, rebuild the
// persistent kernel's lattice list, shared-memory size, occupancy and work list.
int assign_modes(ising_batch *b)
{
    b->h_lats.clear();
    int max_local = 0;
    for (auto &k : b->cls) {
        k.streamed = b->stream_min_L > 0 && k.L >= b->stream_min_L && k.L % 256 == 0;
        k.cfg = default_sweep_config(k.L, k.R);
        if (k.streamed) continue;
        const Geom g = make_geom(k.L);
        for (int r = 0; r < k.R; ++r)
            b->h_lats.push_back(BatchLattice{k.lat + (int64_t)r * 2 * g.nw, k.seed + (uint64_t)r, k.L, 0});
        if (lattice_bytes(k.L) <= 96 * 1024) max_local = std::max<int>(max_local, (int)lattice_bytes(k.L));
    }
    int nstreamed = 0;
    for (const auto &k : b->cls) nstreamed += k.streamed;
    // side streams: one per streamed class (segments) and one per class after the first
    // (measurements)
    const int nside = std::max(nstreamed, (int)b->cls.size() - 1);
    while ((int)b->side.size() < nside) {
        cudaStream_t st = nullptr;
        BCK(b, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->side.push_back(st);
    }
    while ((int)b->ev.size() < nside + 1) {
        cudaEvent_t e = nullptr;
        BCK(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->ev.push_back(e);
    }
    cudaFree(b->d_lats);
    b->d_lats = nullptr;
    if (cudaMalloc(&b->d_lats, sizeof(BatchLattice) * std::max<size_t>(1, b->h_lats.size())) != cudaSuccess)
        return ISING_ENOMEM;
    if (!b->h_lats.empty())
        BCK(b, cudaMemcpyAsync(b->d_lats, b->h_lats.data(), sizeof(BatchLattice) * b->h_lats.size(),
                               cudaMemcpyHostToDevice, b->stream));
    b->smem = max_local;
    BCK(b, batch_occupancy(std::max(b->smem, 0), &b->occ));
    if (b->occ < 1) return bfail(b, ISING_ECUDA, "batch kernel does not fit an SM");
    b->capacity = b->occ * b->sms;
    int s = build_plan(b);
    if (s != ISING_OK) return s;
    return upload_plan(b);
}

}  // namespace

extern "C" {

int ising_batch_set_streamed(ising_batch *b, int min_L)
{
    int s = bcheck(b);
    if (s) return s;
    DevGuard dg(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    b->stream_min_L = min_L;
    return assign_modes(b);
}

int ising_batch_streamed_classes(const ising_batch *b)
{
    if (!b) return -1;
    int n = 0;
    for (const auto &k : b->cls) n += k.streamed;
    return n;
}

int ising_batch_destroy(ising_batch *b)
{
    if (!b) return ISING_OK;
    {
        DevGuard dg(b->device);
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        for (auto &k : b->cls) {
            cudaFree(k.lat);
            cudaFree(k.alt);
            cudaFree(k.xt);
        }
        cudaFree(b->d_lats);
        cudaFree(b->d_tasks);
        cudaFree(b->d_barriers);
        cudaFree(b->d_status);
        cudaFree(b->d_cta_ns);
        cudaFree(b->d_rec);
        cudaFree(b->d_der);
        for (cudaStream_t st : b->side) cudaStreamDestroy(st);
        for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
        if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    }
    delete b;
    return ISING_OK;
}

int ising_batch_create(ising_batch **out, int nclass, const int *L, const int *replicas, const uint64_t *seeds,
                       const ising_opts *opts)
{
    if (!out) return ISING_EINVAL;
    *out = nullptr;
    if (nclass < 1 || !L || !replicas || !seeds) return ISING_EINVAL;
    ising_opts o;
    ising_default_opts(&o);
    if (opts) o = *opts;
    if (o.tie < 0 || o.tie > 2 || o.form != ISING_FORM_PACKED || o.cycle != ISING_CYCLE_01 ||
        o.scheme != ISING_SCHEME_CHECKERBOARD)
        return ISING_EINVAL;
    for (int c = 0; c < nclass; ++c)
        if (!packed_L_ok(L[c]) || L[c] > 4096 || replicas[c] < 1 || replicas[c] > 65535) return ISING_EINVAL;
    ising_batch *b = new (std::nothrow) ising_batch();
    if (!b) return ISING_ENOMEM;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete b;
        return ISING_ECUDA;
    }
    b->device = dev;
    b->rule = o.tie;
    DevGuard dg(dev);
    auto bail = [&](int s) {
        ising_batch_destroy(b);
        return s;
    };
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(ISING_ECUDA);
        b->own_stream = true;
    }
    int64_t rec_off = 0, der_off = 0;
    for (int c = 0; c < nclass; ++c) {
        BatchClass k{L[c], replicas[c], seeds[c], nullptr, rec_off, der_off, 0, SweepConfig{VARIANT_WORD, 0, 0, 0},
                     nullptr, nullptr};
        const int64_t bytes = lattice_bytes(L[c]) * replicas[c];
        if (cudaMalloc(&k.lat, (size_t)bytes) != cudaSuccess) {
            b->cls.push_back(k);
            return bail(ISING_ENOMEM);
        }
        // L >= 512: the correlation sums on the tensor cores, as a single context chooses them
        // (far faster than bit counts there); the scratch is allocated here, never while a
        // schedule is being captured
        if (L[c] >= 512 && corr_mma_supported(L[c]) &&
            cudaMalloc(&k.xt, corr_mma_scratch_bytes(L[c], replicas[c])) != cudaSuccess) {
            k.xt = nullptr;
            cudaFree(k.lat);
            k.lat = nullptr;
            b->cls.push_back(k);
            return bail(ISING_ENOMEM);
        }
        if (L[c] < 64 && cudaMemsetAsync(k.lat, 0, (size_t)bytes, b->stream) != cudaSuccess) return bail(ISING_ECUDA);
        if (launch_init_packed(k.lat, L[c], replicas[c], seeds[c], b->stream) != cudaSuccess) {
            b->cls.push_back(k);
            return bail(ISING_ECUDA);
        }
        b->launches += 1;
        b->cls.push_back(k);
        rec_off += ising_record_len(L[c]) * replicas[c];
        der_off += replicas[c];
    }
    b->nlat = der_off;
    b->rec_words = rec_off;
    if (cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess) return bail(ISING_ECUDA);
    if (cudaMalloc(&b->d_rec, sizeof(int64_t) * (size_t)b->rec_words) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaMalloc(&b->d_der, sizeof(double) * 4 * (size_t)b->nlat) != cudaSuccess) return bail(ISING_ENOMEM);
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return bail(ISING_ECUDA);
    int s = assign_modes(b);
    if (s != ISING_OK) return bail(s);
    *out = b;
    return ISING_OK;
}

int ising_batch_sweep(ising_batch *b, int64_t n)
{
    int s = bcheck(b);
    if (s) return s;
    if (n < 0 || b->t + n > (int64_t)0xffffffffll) return bfail(b, ISING_EINVAL, "bad sweep count");
    if (n == 0) return ISING_OK;
    DevGuard dg(b->device);
    return enqueue_segment(b, n, nullptr);
}

int64_t ising_batch_record_words(const ising_batch *b) { return b ? b->rec_words : -1; }

int64_t ising_batch_lattices(const ising_batch *b) { return b ? b->nlat : -1; }

int ising_batch_measure_ex(ising_batch *b, int64_t *rec, double *derived, double c, unsigned flags)
{
    int s = bcheck(b);
    if (s) return s;
    if (flags & ~(ISING_MEAS_DEVICE | ISING_MEAS_CONNECTED | ISING_MEAS_NO_CORR))
        return bfail(b, ISING_EINVAL, "unknown flags");
    DevGuard dg(b->device);
    const bool dev = flags & ISING_MEAS_DEVICE;
    int64_t *r = (dev && rec) ? rec : b->d_rec;
    double *d = derived ? (dev ? derived : b->d_der) : nullptr;
    if ((s = enqueue_measure(b, r, d, c, flags)) != ISING_OK) return s;
    if (!dev) {
        if (rec)
            BCK(b, cudaMemcpyAsync(rec, r, sizeof(int64_t) * b->rec_words, cudaMemcpyDeviceToHost, b->stream));
        if (derived)
            BCK(b, cudaMemcpyAsync(derived, d, sizeof(double) * 4 * b->nlat, cudaMemcpyDeviceToHost, b->stream));
        return read_status(b);
    }
    return ISING_OK;
}

int ising_batch_run(ising_batch *b, const int64_t *times, int K, int64_t *rec, double *derived, double c,
                    unsigned flags)
{
    int s = bcheck(b);
    if (s) return s;
    if (!times || K < 1 || !rec) return bfail(b, ISING_EINVAL, "bad schedule or output");
    if (flags & ~(ISING_MEAS_DEVICE | ISING_MEAS_CONNECTED | ISING_MEAS_NO_CORR))
        return bfail(b, ISING_EINVAL, "unknown flags");
    int64_t prev = b->t;
    for (int k = 0; k < K; ++k) {
        if (times[k] < prev || times[k] > (int64_t)0xffffffffll) return bfail(b, ISING_EINVAL, "times must not decrease");
        prev = times[k];
    }
    DevGuard dg(b->device);
    const bool dev = flags & ISING_MEAS_DEVICE;
    int64_t *rdst = rec;
    double *ddst = derived;
    std::vector<int64_t *> tmp;
    if (!dev) {
        // device staging for a host result: one record block and derived block per time
        int64_t *r = nullptr;
        double *d = nullptr;
        if (cudaMallocAsync(&r, sizeof(int64_t) * b->rec_words * K, b->stream) != cudaSuccess)
            return bfail(b, ISING_ENOMEM, "staging");
        if (derived && cudaMallocAsync(&d, sizeof(double) * 4 * b->nlat * K, b->stream) != cudaSuccess) {
            cudaFreeAsync(r, b->stream);
            return bfail(b, ISING_ENOMEM, "staging");
        }
        rdst = r;
        ddst = d;
    }
    // key of the cached graph: start time, flags, c, the schedule and the output pointers
    std::vector<int64_t> key = {b->t, (int64_t)flags, (int64_t)std::llround(c * 1e15), (int64_t)(intptr_t)rdst,
                                (int64_t)(intptr_t)ddst, b->missing_cta};
    key.insert(key.end(), times, times + K);
    const int64_t t_start = b->t;
    if (!(b->gexec && key == b->gkey)) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int st = ISING_OK;
        for (int k = 0; k < K && st == ISING_OK; ++k) {
            st = enqueue_segment(b, times[k] - b->t, nullptr);
            if (st == ISING_OK)
                st = enqueue_measure(b, rdst + (int64_t)k * b->rec_words, ddst ? ddst + (int64_t)k * 4 * b->nlat : nullptr,
                                     c, flags);
        }
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        b->t = t_start;
        if (st != ISING_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
        b->gkey = key;
    }
    BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    b->t = times[K - 1];
    if (!dev) {
        BCK(b, cudaMemcpyAsync(rec, rdst, sizeof(int64_t) * b->rec_words * K, cudaMemcpyDeviceToHost, b->stream));
        if (derived)
            BCK(b, cudaMemcpyAsync(derived, ddst, sizeof(double) * 4 * b->nlat * K, cudaMemcpyDeviceToHost, b->stream));
        int st = read_status(b);
        // the cached graph refers to these buffers: drop it with them
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
            b->gkey.clear();
        }
        cudaFreeAsync(rdst, b->stream);
        if (ddst) cudaFreeAsync(ddst, b->stream);
        return st;
    }
    return ISING_OK;
}

int ising_batch_reinit(ising_batch *b)
{
    int s = bcheck(b);
    if (s) return s;
    DevGuard dg(b->device);
    for (const auto &k : b->cls) {
        BCK(b, launch_init_packed(k.lat, k.L, k.R, k.seed, b->stream));
        b->launches += 1;
    }
    b->t = 0;
    return ISING_OK;
}

int ising_batch_get_packed(ising_batch *b, int cls, int replica, uint32_t *words, unsigned flags)
{
    int s = bcheck(b);
    if (s) return s;
    if (cls < 0 || cls >= (int)b->cls.size() || replica < 0 || replica >= b->cls[cls].R || !words ||
        (flags & ~ISING_PTR_DEVICE))
        return bfail(b, ISING_EINVAL, "bad class, replica, buffer or flags");
    DevGuard dg(b->device);
    const auto &k = b->cls[cls];
    const int64_t nw2 = 2 * make_geom(k.L).nw;
    const bool dev = flags & ISING_PTR_DEVICE;
    BCK(b, cudaMemcpyAsync(words, k.lat + (int64_t)replica * nw2, sizeof(uint32_t) * nw2,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (!dev) return read_status(b);
    return ISING_OK;
}

int ising_batch_sync(ising_batch *b)
{
    int s = bcheck(b);
    if (s) return s;
    DevGuard dg(b->device);
    return read_status(b);
}

int ising_batch_get_time(const ising_batch *b, int64_t *t)
{
    if (!b || !t) return ISING_EINVAL;
    *t = b->t;
    return ISING_OK;
}

int ising_batch_plan(const ising_batch *b, int *ntasks, int *nlocal, int *ngroups, int *capacity)
{
    if (!b) return ISING_EINVAL;
    int nl = 0;
    for (const auto &t : b->h_tasks) nl += t.mode == BATCH_LOCAL;
    if (ntasks) *ntasks = (int)b->h_tasks.size();
    if (nlocal) *nlocal = nl;
    if (ngroups) *ngroups = b->ngroups;
    if (capacity) *capacity = b->capacity;
    return ISING_OK;
}

int ising_batch_tune(ising_batch *b, int probe_mcs, double *w_local_out)
{
    int s = bcheck(b);
    if (s) return s;
    if (probe_mcs < 1) return bfail(b, ISING_EINVAL, "probe_mcs must be >= 1");
    DevGuard dg(b->device);
    // Probe rounds: run a short segment, read each CTA's elapsed time, and set the LOCAL
    // weight to the measured ratio of time per spin (LOCAL vs GROUP); rebuild the plan.
    // The probe advances the batch (the state stays a valid trajectory: t moves on).
    for (int round = 0; round < 3 && !b->h_tasks.empty(); ++round) {
        if ((s = enqueue_segment(b, probe_mcs, b->d_cta_ns)) != ISING_OK) return s;
        std::vector<unsigned long long> ns(b->h_tasks.size());
        BCK(b, cudaMemcpyAsync(ns.data(), b->d_cta_ns, sizeof(unsigned long long) * ns.size(), cudaMemcpyDeviceToHost,
                               b->stream));
        if ((s = read_status(b)) != ISING_OK) return s;
        double tl = 0, sl = 0, tg = 0, sg = 0;
        for (size_t i = 0; i < ns.size(); ++i) {
            const BatchTask &t = b->h_tasks[i];
            if (t.mode == BATCH_LOCAL) {
                double spins = 0;
                for (int j = t.first; j < t.first + t.count; ++j) spins += std::pow((double)b->h_lats[j].L, 3);
                tl += (double)ns[i];
                sl += spins;
            } else {
                const double N = std::pow((double)b->h_lats[t.first].L, 3);
                tg += (double)ns[i];
                sg += N / t.size;
            }
        }
        if (sl > 0 && sg > 0 && tg > 0) {
            const double ratio = (tl / sl) / (tg / sg);
            b->w_local = std::max(0.05, std::min(20.0, b->w_local * std::sqrt(ratio * b->w_group / b->w_local)));
        }
        if ((s = build_plan(b)) != ISING_OK) return bfail(b, s, "plan");
        if ((s = upload_plan(b)) != ISING_OK) return s;
    }
    // Streamed classes: candidates are the class's default kernel and the one the single-
    // lattice autotuner picks for its size and replica count alone (timed on scratch
    // contexts).  The streamed classes run side by side within a segment and compete for
    // the SMs, so each class keeps the candidate with which the whole segment (every class)
    // is fastest, one class after the other.
    BCK(b, cudaStreamSynchronize(b->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(b, ISING_ECUDA, "event");
    }
    auto segment_ms = [&](float *ms) -> int {
        int st = enqueue_segment(b, probe_mcs, nullptr);  // warm-up (first launches of a kernel)
        if (st == ISING_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) st = ISING_ECUDA;
        if (st == ISING_OK) st = enqueue_segment(b, 2 * (int64_t)probe_mcs, nullptr);
        if (st == ISING_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
            st = ISING_ECUDA;
        if (st == ISING_OK) st = read_status(b);
        return st;
    };
    for (int c = 0; c < (int)b->cls.size() && s == ISING_OK; ++c) {
        if (!b->cls[c].streamed) continue;
        ising_opts base, alone, dflt;
        ising_default_opts(&base);
        base.tie = (ising_tie)b->rule;
        base.device = b->device;
        dflt = base;
        if (ising_tune_sweep(b->cls[c].L, b->cls[c].R, probe_mcs, &base, &alone, nullptr) != ISING_OK) {
            s = bfail(b, ISING_ECUDA, "tuning a streamed class");
            break;
        }
        float ms_dflt = 0.f, ms_alone = 0.f;
        if ((s = ising_batch_set_class_opts(b, c, &dflt)) != ISING_OK || (s = segment_ms(&ms_dflt)) != ISING_OK ||
            (s = ising_batch_set_class_opts(b, c, &alone)) != ISING_OK || (s = segment_ms(&ms_alone)) != ISING_OK)
            break;
        if (ms_dflt <= ms_alone) s = ising_batch_set_class_opts(b, c, &dflt);
    }
    // the streamed classes beside the persistent launch, or after it
    if (s == ISING_OK && !b->h_tasks.empty() && ising_batch_streamed_classes(b) > 0) {
        float ms_after = 0.f, ms_beside = 0.f;
        if ((s = ising_batch_set_overlap(b, 0)) == ISING_OK && (s = segment_ms(&ms_after)) == ISING_OK &&
            (s = ising_batch_set_overlap(b, 1)) == ISING_OK && (s = segment_ms(&ms_beside)) == ISING_OK &&
            ms_after <= ms_beside)
            s = ising_batch_set_overlap(b, 0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ISING_OK) return s;
    if (w_local_out) *w_local_out = b->w_local;
    return ISING_OK;
}

int ising_batch_set_class_opts(ising_batch *b, int cls, const ising_opts *o)
{
    int s = bcheck(b);
    if (s) return s;
    if (!o || cls < 0 || cls >= (int)b->cls.size()) return bfail(b, ISING_EINVAL, "bad class");
    BatchClass &k = b->cls[cls];
    if (!k.streamed) return bfail(b, ISING_EINVAL, "class is swept by the persistent kernel");
    SweepConfig cfg{};
    if (!resolve_sweep_config(k.L, k.R, o->variant, o->tile_y, o->tile_z, o->depth, &cfg))
        return bfail(b, ISING_EINVAL, "sweep configuration not valid for this L");
    DevGuard dg(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    if (cfg.variant == VARIANT_ZFUSE && !k.alt &&
        cudaMalloc(&k.alt, (size_t)(lattice_bytes(k.L) * k.R)) != cudaSuccess) {
        k.alt = nullptr;
        return bfail(b, ISING_ENOMEM, "second store of the fused sweep");
    }
    k.cfg = cfg;
    if (b->gexec) {  // the cached schedule graph holds the old kernels
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->gkey.clear();
    }
    return ISING_OK;
}

int ising_batch_set_overlap(ising_batch *b, int on)
{
    int s = bcheck(b);
    if (s) return s;
    if (on != 0 && on != 1) return bfail(b, ISING_EINVAL, "overlap must be 0 or 1");
    DevGuard dg(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    b->overlap = on;
    if (b->gexec) {  // the cached schedule graph holds the old stream order
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->gkey.clear();
    }
    return ISING_OK;
}

int ising_batch_overlap(const ising_batch *b) { return b ? b->overlap : -1; }

int ising_batch_get_class_opts(const ising_batch *b, int cls, ising_opts *o)
{
    if (!b || !o || cls < 0 || cls >= (int)b->cls.size()) return ISING_EINVAL;
    const BatchClass &k = b->cls[cls];
    ising_default_opts(o);
    o->variant = k.streamed ? k.cfg.variant : -1;
    o->tile_y = k.cfg.tile_y;
    o->tile_z = k.cfg.tile_z;
    o->depth = k.cfg.depth;
    return ISING_OK;
}

int ising_batch_set_weights(ising_batch *b, double w_local, double w_group)
{
    int s = bcheck(b);
    if (s) return s;
    if (!(w_local > 0) || !(w_group > 0)) return bfail(b, ISING_EINVAL, "weights must be > 0");
    DevGuard dg(b->device);
    b->w_local = w_local;
    b->w_group = w_group;
    if ((s = build_plan(b)) != ISING_OK) return bfail(b, s, "plan");
    return upload_plan(b);
}

int ising_batch_inject_missing_cta(ising_batch *b, int cta, double timeout_s)
{
    if (!b) return ISING_EINVAL;
    if (cta < -1 || cta >= (int)b->h_tasks.size() || !(timeout_s > 0)) return bfail(b, ISING_EINVAL, "bad injection");
    b->missing_cta = cta;
    b->timeout_ns = (uint64_t)(timeout_s * 1e9);
    return ISING_OK;
}

const char *ising_batch_last_error(const ising_batch *b) { return b ? b->err : "null batch"; }

int64_t ising_batch_launch_count(const ising_batch *b) { return b ? b->launches : -1; }

}  // extern "C"
