/*
 * ising.h — C ABI of the GB300 zero-temperature checkerboard quench library.
 *
 * The library simulates the quench studied in Gessert, Christiansen, Janke,
 * "Superdiffusion-like behavior in zero-temperature coarsening of the d=3 Ising model"
 * (arXiv:2305.12161): a periodic simple-cubic L^3 nearest-neighbour Ising model
 * (H = -sum_<ij> s_i s_j) started from an infinite-temperature configuration and
 * evolved with single-spin flips under the T -> 0 Glauber acceptance (Eq. 6: dE < 0
 * always, dE > 0 never, dE = 0 with probability 1/2), proposals ordered by the
 * checkerboard decomposition (Methods, "Checkerboard update": all red sites, x+y+z
 * even, at once, then all blue sites).  One Monte Carlo sweep (MCS) is both halves.
 * Observables are the integer magnetisation, broken-bond count and the axis
 * correlation sums behind Eq. (2).
 *
 * Conventions shared by every entry point
 *   - Every function returns an ising_status (0 = ISING_OK, negative = error) unless
 *     stated otherwise.  Nothing is thrown across the ABI.
 *   - A context (ising_ctx) owns all device memory of its replicas.  The caller owns
 *     every host buffer, every device buffer it passes in, and the CUDA stream.
 *   - Work is enqueued on the context's stream (a cudaStream_t given at creation, or a
 *     stream the library creates).  Functions that write host memory synchronise that
 *     stream before returning; the others return once the work is enqueued.
 *   - A CUDA error or a device-side timeout poisons the context: every later call
 *     except ising_destroy / ising_strerror / ising_last_error returns ISING_EPOISONED.
 *   - Site (x,y,z), 0 <= x,y,z < L, has linear index i = x + L*(y + L*z) (64-bit).
 *     Sublattice q = (x+y+z) mod 2; q = 0 ("red") is updated first in every sweep.
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11).  The bit of a site of
 *     sublattice q is bit (h & 31) of output word ((h >> 5) & 3) of
 *     Philox(counter = (h >> 7, t, phase, 0), key = (lo32(S), hi32(S))) with
 *     h = (x >> 1) + (L/2)*(y + L*z), S = seed + replica (mod 2^64), phase = q for the
 *     zero-energy decision of sweep t (0-based), phase = 2 + q for the initial state.
 *     A run is therefore reproducible bit for bit and independent of launch shapes.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ising_ctx ising_ctx;

typedef enum {
    ISING_OK = 0,
    ISING_EINVAL = -1,    /* bad argument (size, pointer, replica index, flag) */
    ISING_ENOMEM = -2,    /* device or host allocation failed */
    ISING_ECUDA = -3,     /* a CUDA call failed; the context is poisoned */
    ISING_ETIMEOUT = -4,  /* a bounded device-side wait gave up; the context is poisoned */
    ISING_EBUSY = -5,     /* resource in use (e.g. a batch already running) */
    ISING_EPOISONED = -6  /* an earlier error poisoned this context */
} ising_status;

/* Zero-energy (u = 3 up neighbours) rule.  GLAUBER is the paper's (Eq. 6). */
typedef enum {
    ISING_TIE_GLAUBER = 0, /* flip iff the site's Philox bit is 1 (probability 1/2) */
    ISING_TIE_ALWAYS = 1,  /* always flip: T -> 0 limit of Metropolis, min(1, e^0) */
    ISING_TIE_NEVER = 2    /* never flip */
} ising_tie;

/* Storage form.  PACKED: 1 bit per spin, each sublattice in its own array (the fast
 * form).  PLAIN: one signed byte per spin, one kernel launch per lattice and
 * half-sweep (the comparison form).  Both produce identical spins and records. */
typedef enum { ISING_FORM_PACKED = 0, ISING_FORM_PLAIN = 1 } ising_form;

typedef struct {
    int tie;        /* ising_tie */
    int form;       /* ising_form */
    void *stream;   /* cudaStream_t to enqueue on; NULL: the library creates one */
    int device;     /* CUDA device ordinal; -1: the current device */
    int variant;    /* packed sweep kernel variant, 0 = automatic (see ising_variants):
                       1 one thread per word (any L), 2 z-marching tiles (L multiple of 256),
                       3 z-marching specialised on the row width (L = 256, 512, 1024, 2048),
                       4 as 3 with a deeper copy pipeline and fewer registers,
                       5 one launch per sweep updating both sublattices (L = 256 .. 2048, powers
                         of two; holds a second packed store of the same size, the two swap
                         roles every sweep, so a CUDA graph captured around ising_sweep replays
                         correctly only for an even sweep count) */
    int tile_y;     /* packed z-marching variant: rows per tile (0 = automatic); variant 3
                       (z-marching specialised on the row width) fixes it to 256/(L/256) */
    int tile_z;     /* packed z-marching variants: planes per tile (0 = automatic) */
    int depth;      /* variant 4: planes in flight in the copy pipeline, 2..4 (0 = 3);
                       variant 5: copy groups in flight, 1..3 (0 = 2), plus 8 for tiles of
                       256/(L/256) - 2 rows whose halo rows are computed by ordinary threads,
                       plus 16 for z-blocks fitted to the CTAs resident on the device (tile_z
                       is then their nominal depth); any other value is ISING_EINVAL */
    int cycle;      /* ising_cycle: sublattice order of each sweep */
    int corr;       /* ising_corr: how the correlation sums D_a(r) are computed */
    int scheme;     /* ising_scheme: checkerboard or double checkerboard */
    int block_x;    /* double checkerboard: block sides in sites (0 = default: block_x = L, */
    int block_y;    /*   block_y = 16, block_z = 8, both L when L <= 16); see ising_scheme */
    int block_z;
    int pdl;        /* 1 (ising_default_opts): the z-marching (variant 3) and whole-sweep
                       (variant 5) kernels are launched with programmatic dependent launch:
                       a sweep's CTAs are scheduled while the previous one drains and wait
                       for its completion before they touch memory (same results, shorter
                       gaps between the launches of one stream); 0: plain stream order,
                       which leaves the SMs of a draining kernel to other streams (many
                       contexts sharing the GPU); any other value is ISING_EINVAL */
} ising_opts;

/* Method of the correlation sums (identical results).  POPCOUNT: XOR + bit counts over
 * packed words, any L.  TENSOR: D_a(r) = N/2 - (1/2) sum_j G[j][j+r] with G the Gram
 * matrix of the L positions over the L^2 lines of the axis, computed on the 5th-generation
 * tensor cores (tcgen05.mma, e4m3 operands loaded by TMA, fp32 accumulators in tensor memory;
 * exact: |G| <= L^2 <= 2^24); L a multiple of 128 in 256..2048; it allocates a scratch of
 * 2 L^3 bytes (two axes of one replica expanded to e4m3, one multiplied while the next is
 * expanded: 17.2 GB at L=2048) at its first use and keeps it (ising_release_scratch frees it).  AUTO:
 * TENSOR for L >= 512 where it is supported and its scratch can be allocated (measured on
 * GB300: 1.9x faster than POPCOUNT at L=512, 3.5x at L=2048; slower at L=256), else POPCOUNT. */
typedef enum { ISING_CORR_AUTO = 0, ISING_CORR_POPCOUNT = 1, ISING_CORR_TENSOR = 2 } ising_corr;

/* Sublattice order of a sweep.  01: red (q = 0) then blue every sweep (the paper's main
 * runs, Methods).  MIXED: the first sublattice of each sweep is random (Supp. Methods I B,
 * the "mixed cycle" that restores detailed balance): sweep t of the lattice keyed S goes
 * blue first when bit 0 of word 0 of Philox(counter (0, t, 5, 0), key S) is 1.  With
 * replicas > 1 each replica draws its own order (the half-sweep kernels launch once per
 * replica and half-sweep; the whole-sweep kernel carries each replica's order in its
 * parameters).  The batched form supports the 01 cycle only. */
typedef enum { ISING_CYCLE_01 = 0, ISING_CYCLE_MIXED = 1 } ising_cycle;

/* Update scheme of a sweep.  CHECKERBOARD: the two half-sweeps of the main text (Methods).
 * DOUBLE: the double-checkerboard decomposition (Supp. Methods I A, Weigel's GPU scheme in
 * d = 3).  The lattice is cut into blocks of block_x * block_y * block_z sites; block
 * (i, j, k) = (x / block_x, y / block_y, z / block_z) is red when i + j + k is even.  A
 * sweep updates all red blocks, then all blue ones; inside a block the sites of odd
 * parity (x + y + z) first, then the even ones (the step list's "darker" sites first).
 * With ISING_CYCLE_MIXED (Supp. Methods I B) the colour order is drawn per sweep and
 * replica as for the checkerboard, and the parity each block starts with per block and
 * sweep: block beta = i + nbx*(j + nby*k) starts with parity 1 when bit (beta & 31) of
 * word ((beta >> 5) & 3) of Philox(counter (beta >> 7, t, 6, 0), key S) is 1.  A site's
 * zero-energy decision uses the checkerboard's bit (phase = its parity), so 1x1x1 blocks
 * give exactly the checkerboard sweep.  Requirements (else ISING_EINVAL at creation):
 * PACKED form; block_y and block_z divide L with an even quotient (or equal L); block_x
 * equals L, or (L >= 128) is a multiple of 64 dividing L with an even quotient; a block
 * with a one-row halo on each side must fit in 227 KB of shared memory,
 * 8 * (block_y + 2) * (block_z + 2) * (row words) bytes with row words = L/64 (1 for
 * L < 64) when block_x = L, else block_x/64 + 8 when block_x is a multiple of 256 and
 * block_x/64 + 2 otherwise.
 * Not available in the batched form. */
typedef enum { ISING_SCHEME_CHECKERBOARD = 0, ISING_SCHEME_DOUBLE = 1 } ising_scheme;

/* Fill *opts with the defaults: GLAUBER, PACKED, own stream, current device, auto. */
void ising_default_opts(ising_opts *opts);

/* Create R = `replicas` independent lattices of linear size L, replica r seeded with
 * S = seed + r, each in its T = infinity initial state (t = 0; Results and Discussion:
 * random configurations with m ~ 0, drawn here i.i.d. with probability 1/2).
 * L must be even and >= 4; the PACKED form additionally needs L a multiple of 64 or
 * L in {4, 8, 16, 32}.  On success *out receives the context; on error *out = NULL. */
int ising_create(ising_ctx **out, int L, int replicas, uint64_t seed);
int ising_create_ex(ising_ctx **out, int L, int replicas, uint64_t seed, const ising_opts *opts);

/* Device bytes that a context of `replicas` lattices of size L with options *opts (NULL:
 * defaults) holds once it has measured (no counterpart in the paper: it serves admission by
 * device footprint, e.g. the serving loop's): the packed store (2 x L^3/16 bytes per replica,
 * twice for the fused whole-sweep kernel, variant 5), the byte-per-spin lattice of the
 * PLAIN form (L^3 per replica), the records and derived values, and the tensor-core
 * correlation scratch (2 L^3 bytes, allocated by the first measurement whose method is the
 * tensor-core path: ISING_CORR_TENSOR, or AUTO with L >= 512).  Pure host arithmetic,
 * no device is touched; what ising_create_ex allocates comes from the same accounting.
 * Not included: buffers that only the optional calls allocate while they run or keep
 * (get/set_spins stage L^3 bytes for the duration of the call; ising_measure_radial keeps
 * its FFT buffer and ISING_PTR_HOST_ASYNC its staging copy until ising_release_scratch).
 * Returns -1 for arguments that ising_create_ex would refuse. */
int64_t ising_footprint_bytes(int L, int replicas, const ising_opts *opts);

/* Redraw every replica's T = infinity initial state for a new seed (replica r uses
 * seed + r) and reset t to 0, reusing the context's memory.  Enqueued, no sync. */
int ising_reinit(ising_ctx *ctx, uint64_t seed);

/* Replace every replica's state by a Menger-sponge start (Results, the sponge test):
 * tiles of k-th-iteration sponges of side 3^k (cut at the lattice edge), a cell in the
 * sponge unless at some base-3 digit position two or three of its coordinates' digits
 * are 1; sponge cells take the tile's random sign, removed cells the opposite.  Tile
 * T = tx + nT*(ty + nT*tz), nT = ceil(L/3^k), is +1 when bit (T & 31) of word
 * ((T >> 5) & 3) of Philox(counter (T >> 7, 0, 4, 0), key seed + replica) is 1.
 * k = 0..8; resets t to 0.  Enqueued, no sync. */
int ising_init_menger(ising_ctx *ctx, int k);

/* Enqueue n_mcs >= 0 Monte Carlo sweeps on every replica (each sweep: red half-sweep,
 * then blue half-sweep; Methods, "Checkerboard update").  Advances the context's
 * time t by n_mcs.  Returns once the work is enqueued. */
int ising_sweep(ising_ctx *ctx, int64_t n_mcs);

/* ---- Radially averaged three-dimensional correlation and structure factor ----------
 * (Methods, "Calculating the correlation function": the spin-spin sum over every lag
 * vector k, G(k) = sum_i s_i s_(i+k), from two FFTs, Eq. (3), then averaged radially;
 * Results: the structure factor S(k,t), the Fourier transform of C.)
 * Lag and mode components are minimal images (j <= L/2: j, else j - L); a vector of squared
 * length D falls in bin b = round(sqrt(D)) = (isqrt(4D) + 1) / 2, b = 0 .. nbins-1 with
 * nbins = ising_radial_bins(L) = round(sqrt(3) L / 2) + 1; bins beyond L/2 are cut by the
 * cube's corners.
 *   C[b] = (sum of G(k) over the bin's lags) / (N * count[b])
 *   S[b] = (sum of |FFT(s)(q)|^2 over the bin's modes) / (N * count[b]), wave number 2 pi b / L
 *   *ell = the radial C's first downward crossing of cval for r <= L/2, linearly
 *          interpolated (NaN if none)
 * count[b] is the number of lag (= mode) vectors in the bin.  G(k) is an integer: the
 * library rounds every FFT value g/N to the nearest integer before summing, so C is exact
 * whenever the FFT error stays below 1/2; *inexact receives the number of lags whose value lay
 * more than 1/4 from an integer (0: C is exact).  precision: ISING_FFT_SINGLE (fp32 cuFFT;
 * exact at small L, within the rounding error of single-precision FFTs at large L) or
 * ISING_FFT_DOUBLE (fp64 cuFFT: exact up to L = 2048 at least; S to fp64 rounding).  Host
 * outputs: C and S of nbins doubles (required), count of nbins int64, ell, inexact (each may
 * be NULL).  Replica `replica` only.  The first call allocates, in stream order,
 * L^2 (L/2+1) complex values of the chosen precision (34.4 GB at L=2048 in single
 * precision, twice that in double) plus cuFFT's work area, and keeps them in the context for
 * later calls (ising_release_scratch frees them); ISING_ENOMEM (context still usable) if the
 * device has no room.  Synchronises the context's stream.  ising_radial_bins returns -1 for a
 * bad L. */
typedef enum { ISING_FFT_SINGLE = 0, ISING_FFT_DOUBLE = 1 } ising_fft_precision;
int64_t ising_radial_bins(int L);
int ising_measure_radial(ising_ctx *ctx, int replica, int precision, double cval, double *C, double *S,
                         int64_t *count, double *ell, int64_t *inexact);
/* Failure injection for tests: the next measurement that runs on the tensor cores loses one
 * operand load in one CTA, so that CTA's bounded wait for it runs out after timeout_s
 * (0 < timeout_s <= 60; it also becomes the bound of every later device-side wait of the
 * context); the kernel gives up, releases its tensor memory and sets the context's error
 * flag, and the synchronising call returns ISING_ETIMEOUT (the context is then poisoned).
 * No fault is raised on the device. */
int ising_inject_corr_stall(ising_ctx *ctx, double timeout_s);

/* Free the scratch that measurements keep in the context (the radial measurement's transform
 * buffer and work area, the tensor-core correlation's expanded lattice) and the staging
 * buffer of asynchronous ising_set_packed; the next call that needs one allocates it again.
 * Synchronises the context's streams. */
int ising_release_scratch(ising_ctx *ctx);

/* Number of int64 values of one replica's record:
 *   [t, M, B, D_x(0..L/2), D_y(0..L/2), D_z(0..L/2)]  -> 3 + 3*(L/2 + 1),
 * t = completed MCS, M = sum_i s_i, B = number of unequal nearest-neighbour pairs
 * (E = -(3N - 2B)), D_a(r) = #{ i : s_i != s_(i + r e_a) }.  Returns -1 for bad L. */
int64_t ising_record_len(int L);

/* Measure every replica and write replicas * ising_record_len(L) int64 values to the
 * HOST buffer `out` (replica-major).  Synchronises the context's stream. */
int ising_measure(ising_ctx *ctx, int64_t *out);

/* Flags of ising_measure_ex. */
#define ISING_MEAS_DEVICE 1u    /* rec / derived are device pointers; do not synchronise */
#define ISING_MEAS_CONNECTED 2u /* derived l_C uses C(r) - m^2 (second term of Eq. 2) */
#define ISING_MEAS_NO_CORR 4u   /* skip D_a(r) (they are written as -1): energy and m only */

/* Measure into `rec` (replicas * record_len int64, may be NULL) and, if `derived` is
 * not NULL, write per replica 4 doubles [e, m, l_E, l_C]:
 *   e = -3 + 2B/N, m = M/N, l_E = N/B (+inf when B = 0),
 *   l_C = first intersection of C(r) = sum_a (N - 2 D_a(r)) / (3N) with the constant
 *   c (Results: c = 0.5), linearly interpolated; NaN if C does not cross c, r <= L/2.
 * Without ISING_MEAS_DEVICE both pointers are host memory and the call synchronises. */
int ising_measure_ex(ising_ctx *ctx, int64_t *rec, double *derived, double c, unsigned flags);

/* Copy one replica's spins to / from a HOST int8 buffer of N = L^3 values (+1 / -1)
 * indexed x + L*(y + L*z).  ising_set_spins rejects values other than +-1 with
 * ISING_EINVAL (checked on the host before anything is copied).  Both synchronise. */
int ising_get_spins(ising_ctx *ctx, int replica, int8_t *host_out);
int ising_set_spins(ising_ctx *ctx, int replica, const int8_t *host_in);

/* Flags of the packed-state calls. */
#define ISING_PTR_DEVICE 1u /* the buffer is device memory; no synchronisation */
/* ising_set_packed only: the host buffer is page-locked (cudaHostAlloc / registered) and the
 * caller keeps it alive and unchanged until ising_sync returns.  The call returns without
 * waiting: the words go to a staging buffer of the context (one replica's packed size,
 * allocated on first use, freed by ising_release_scratch or ising_destroy) on a copy stream
 * of its own, so the transfer overlaps work already queued on the context's stream; that
 * stream then waits for it and copies the staged words into the replica.  Ordering with the
 * context's other calls is as for ISING_PTR_DEVICE. */
#define ISING_PTR_HOST_ASYNC 2u

/* Number of uint32 words of one replica's packed state (2 * ceil(N/64) style, see
 * below); -1 for bad L.  Layout: sublattice 0 then sublattice 1; within a sublattice,
 * bit j of word w is the site with compressed index h = 32*w + j (1 = up) for
 * L a multiple of 64; for L < 64 each row (y,z) has its own word holding its L/2 sites
 * in bits 0..L/2-1.  This is the checkpoint format: with (seed, t) it resumes a run
 * bit for bit. */
int64_t ising_packed_words(int L);
int ising_get_packed(ising_ctx *ctx, int replica, uint32_t *words, unsigned flags);
int ising_set_packed(ising_ctx *ctx, int replica, const uint32_t *words, unsigned flags);

/* Completed-sweep counter t shared by all replicas of the context. */
int ising_get_time(ising_ctx *ctx, int64_t *t);
int ising_set_time(ising_ctx *ctx, int64_t t);

/* Block until the context's stream is idle; reports asynchronous errors. */
int ising_sync(ising_ctx *ctx);

/* Release the context and its device memory.  NULL-safe.  Always returns ISING_OK for
 * a valid or NULL pointer. */
int ising_destroy(ising_ctx *ctx);

/* Static message for a status code. */
const char *ising_strerror(int status);

/* Detail of the last error recorded on the context (empty string if none). */
const char *ising_last_error(const ising_ctx *ctx);

/* Number of kernel launches this context has enqueued so far (diagnostics). */
int64_t ising_launch_count(const ising_ctx *ctx);

/* ---------------------------------------------------------------------------------
 * Batched form: many independent lattices of uneven L in one context.  Class c holds
 * replicas[c] lattices of size L[c], replica r seeded seeds[c] + r, each in its
 * T = infinity start; all share the sweep counter t.  A segment of n MCS is ONE
 * persistent cooperative kernel launch over a CTA work list: lattices small enough
 * for one CTA's shared memory (e.g. 64^3 = 32 KiB packed) are owned whole by one CTA
 * and swept there; larger ones are split into slabs over a group of CTAs that meet at
 * a bounded barrier in global memory between half-sweeps.  Classes with L a multiple of
 * 256 and at least the streaming threshold (default 256; ising_batch_set_streamed) are
 * instead swept in the same segment by a single-lattice sweep kernel (the z-marching one
 * by default, the one ising_batch_tune picks after tuning), which streams them faster
 * than slab groups do.  Every lattice follows
 * exactly the trajectory of the single-lattice entry points (same rule, order and
 * random bits), so batching changes speed, not results.
 * Records and derived values are concatenated in class order, replica-major within a
 * class: ising_batch_record_words() int64 and 4 * ising_batch_lattices() doubles per
 * measured time; a measurement runs one class per stream, and classes with L >= 512 take
 * their correlation sums on the tensor cores (identical results), for which
 * ising_batch_create allocates 2 L^3 bytes of scratch per such class.  Only the PACKED
 * form is batched (opts->form must be PACKED). */
typedef struct ising_batch ising_batch;
int ising_batch_create(ising_batch **out, int nclass, const int *L, const int *replicas, const uint64_t *seeds,
                       const ising_opts *opts);
/* Enqueue n_mcs sweeps of every lattice: one persistent launch (per 2^30 sweeps). */
int ising_batch_sweep(ising_batch *b, int64_t n_mcs);
int64_t ising_batch_record_words(const ising_batch *b);
int64_t ising_batch_lattices(const ising_batch *b);
/* Measure every lattice (flags as ising_measure_ex).  Host buffers synchronise and
 * report a barrier timeout of an earlier segment as ISING_ETIMEOUT. */
int ising_batch_measure_ex(ising_batch *b, int64_t *rec, double *derived, double c, unsigned flags);
/* Run a measurement schedule: for k = 0..K-1 sweep to absolute time times[k]
 * (non-decreasing, >= current t) and measure into slot k of rec (K x record_words) and,
 * if not NULL, derived (K x 4 x lattices).  The whole schedule (segments and
 * measurements) is captured into one CUDA graph, which is cached and replayed while the
 * start time, schedule, flags and output pointers repeat.  ISING_MEAS_DEVICE: device
 * outputs, no synchronisation; otherwise host outputs and the call synchronises. */
int ising_batch_run(ising_batch *b, const int64_t *times, int K, int64_t *rec, double *derived, double c,
                    unsigned flags);
/* Redraw every lattice's T = infinity start (same seeds) and reset t to 0. */
int ising_batch_reinit(ising_batch *b);
int ising_batch_get_packed(ising_batch *b, int cls, int replica, uint32_t *words, unsigned flags);
int ising_batch_sync(ising_batch *b);
int ising_batch_get_time(const ising_batch *b, int64_t *t);
/* Work list summary: CTAs, CTAs owning whole lattices, slab groups, co-resident CTAs. */
int ising_batch_plan(const ising_batch *b, int *ntasks, int *nlocal, int *ngroups, int *capacity);
/* Autotuner: probe rounds of probe_mcs sweeps (they advance the batch) time every CTA,
 * set the relative cost of whole-lattice CTAs from the measured time per spin and
 * rebuild the work list; *w_local_out receives the chosen weight.  Then every streamed
 * class, one after the other, keeps whichever of its default kernel and the kernel that
 * ising_tune_sweep picks for its L and replica count alone gives the faster whole segment
 * (the streamed classes of a segment run side by side on their own streams, forked from
 * and joined back into the batch's stream, so they compete for the SMs); last, it keeps
 * the faster of the streamed classes beside or after the persistent launch
 * (ising_batch_set_overlap). */
int ising_batch_tune(ising_batch *b, int probe_mcs, double *w_local_out);
/* Sweep kernel of streamed class `cls` (Methods, "Checkerboard update"; every choice gives
 * the same trajectory): opts->variant, tile_y, tile_z and depth as for ising_create_ex,
 * variant 0 = the default for the class's L and replica count; the other fields are
 * ignored.  Variant 5 (both sublattices per launch, up to 16 replicas of the class per
 * launch) allocates a second store of the class's size, kept until ising_batch_destroy;
 * a segment then runs its whole sweeps in pairs between the two stores and an odd last
 * sweep in place, so the state is always in the first store between segments.
 * ISING_EINVAL: class out of range, not streamed, or a configuration not valid for its L;
 * ISING_ENOMEM: the second store could not be allocated.  Drops the cached schedule graph.
 * ising_batch_set_streamed puts every streamed class back on its default kernel. */
int ising_batch_set_class_opts(ising_batch *b, int cls, const ising_opts *opts);
/* The sweep kernel of class `cls` into opts (variant -1: the class is swept by the
 * persistent kernel); ISING_EINVAL for a bad class or NULL pointer. */
int ising_batch_get_class_opts(const ising_batch *b, int cls, ising_opts *opts);
/* on = 1: within a segment the streamed classes run beside the persistent launch (every one
 * on a side stream forked before it); on = 0 (the default): after it.  The lattices of the
 * two parts are disjoint, so the results are the same either way; ising_batch_tune keeps the
 * faster.  ISING_EINVAL unless on is 0 or 1.  Drops the cached schedule graph. */
int ising_batch_set_overlap(ising_batch *b, int on);
/* The current setting of ising_batch_set_overlap (-1 for a NULL batch). */
int ising_batch_overlap(const ising_batch *b);
int ising_batch_set_weights(ising_batch *b, double w_local, double w_group);
/* Classes with L >= min_L and L % 256 == 0 are swept by a single-lattice kernel, the
 * others by the persistent kernel; min_L <= 0 puts every class in the persistent kernel.
 * Rebuilds the work list (results are unchanged). */
int ising_batch_set_streamed(ising_batch *b, int min_L);
/* Number of classes currently swept by a single-lattice kernel. */
int ising_batch_streamed_classes(const ising_batch *b);
/* Failure injection for tests: CTA `cta` returns at once, so its slab group's barrier
 * waits run out after timeout_s; the segment then ends early and the next
 * synchronising call returns ISING_ETIMEOUT (the batch is poisoned).  cta = -1 clears. */
int ising_batch_inject_missing_cta(ising_batch *b, int cta, double timeout_s);
const char *ising_batch_last_error(const ising_batch *b);
int64_t ising_batch_launch_count(const ising_batch *b);
int ising_batch_destroy(ising_batch *b);

/* Measurement for callers that cannot allocate device memory (no counterpart in the
 * paper; it serves library users).  Some callers may not call cudaMalloc where they
 * measure: code whose device memory is all owned by another allocator or a fixed
 * arena, or code that must not let an allocation synchronise the device mid-pipeline.
 * This entry point allocates nothing: the caller passes the packed lattices (device
 * memory, `replicas` consecutive states in the ising_get_packed layout) and a device
 * output `derived` of replicas x 4 doubles [e, m, l_E, l_C] (as in ising_measure_ex,
 * with the same flags; ISING_MEAS_DEVICE is implied, accepted and ignored).  The integer
 * records it builds on the way live in one fixed array inside the library's device
 * image, ISING_NOALLOC_MAX_RECORD_WORDS int64 (1 MiB), which every GPU that loads the
 * library holds until the process exits.
 *   - Returns ISING_EINVAL when replicas * ising_record_len(L) exceeds that maximum
 *     (e.g. L = 2048 allows 42 replicas), or for a bad L, pointer or flag.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream);
 *     nothing is synchronised.
 *   - The first call on a device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.
 *   - Every call shares the one array, and it keeps the last call's contents (each call
 *     rewrites what it uses before reading it).  Calls that overlap on the GPU (other
 *     streams, other host threads) race on it: order them on one stream. */
#define ISING_NOALLOC_MAX_RECORD_WORDS 131072
int ising_measure_derived_noalloc(const uint32_t *lattice, int L, int replicas, double c, unsigned flags,
                                  double *derived, void *stream);

/* Autotuner of the single-lattice sweep: for `replicas` lattices of size L, times
 * probe_mcs sweeps (after 2 warm-up sweeps) of every valid kernel variant and tile
 * shape (tile_y rows x tile_z planes per CTA; tile_z sets how many 128-spin words each
 * thread updates per launch), on scratch contexts built from *base (NULL: defaults),
 * and writes the fastest options to *best (and its time per MCS in ms).  Variant 5
 * holds a second packed store, so it is chosen only when it beats the fastest
 * single-store candidate by more than 3%.  All candidates give bit-identical results,
 * so the choice affects speed and memory only. */
int ising_tune_sweep(int L, int replicas, int probe_mcs, const ising_opts *base, ising_opts *best,
                     double *best_ms_per_mcs);

/* Packed sweep kernel variants: fills up to `cap` ids into `ids`, returns the number.
 * Every variant produces bit-identical results; they differ in speed only. */
int ising_variants(int *ids, int cap);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */
