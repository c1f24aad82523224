// Host-side launch wrappers of the library's kernels.  Every wrapper enqueues on
// `stream` and returns cudaGetLastError() of its launch(es).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

// ---- packed form: lat points at replica 0; replica r's sublattice q starts at
//      lat + (2*r + q) * nw. -------------------------------------------------------
cudaError_t launch_init_packed(uint32_t *lat, int L, int R, uint64_t seed, cudaStream_t s);

// Packed sweep variants (bit-identical results).
enum SweepVariant : int {
    VARIANT_AUTO = 0,
    VARIANT_WORD = 1,    // one thread per 32-bit word, any supported L
    VARIANT_ZMARCH = 2,  // z-marching, cp.async-staged tiles, 128 spins per thread, L >= 256
    VARIANT_ZFAST = 3,   // z-marching specialised on the row width (L = 256, 512, 1024, 2048)
    VARIANT_ZDEEP = 4,   // as ZFAST with a deeper copy pipeline (depth 2..4) and fewer registers
    VARIANT_ZFUSE = 5,   // one launch per sweep (both sublattices), ping-pong between two stores
};

struct SweepConfig {
    int variant;
    int tile_y;  // rows per tile (z-march; ZFAST: fixed to 256 / (L/256))
    int tile_z;  // planes per tile (z-march)
    int depth;   // ZDEEP: planes in flight beyond the one consumed (2..4)
    int pdl = 1; // ZFAST, ZFUSE: programmatic dependent launch (0: plain stream order)
};

bool sweep_config_valid(int L, const SweepConfig &c);
SweepConfig default_sweep_config(int L, int R);
bool resolve_sweep_config(int L, int R, int variant, int tile_y, int tile_z, int depth, SweepConfig *out);

// Fused sweeps (VARIANT_ZFUSE): each sweep reads *cur and writes *nxt, then swaps the two
// pointers, so after n sweeps *cur holds the state.  Both stores hold 2*R*nw words.
// depth: copy groups in flight while a step computes, 1..3 (0 = 2; SweepConfig.depth); +8 selects
// the balanced tiling (tiles of 256/(L/256) - 2 rows, the halo rows computed by ordinary threads;
// 2 or 3 groups); +16 fits the number of z-blocks (tiles of nearly equal depth, within 25% of
// tile_z) to the resident CTAs so that the launch's last wave is nearly full.  The five-slot
// forms (depth 0, 2, 8, 10 with or without +16) take up to 16 replicas per launch, the others
// one; every replica has its own first sublattice under the mixed cycle.  The kernel bounds
// its waits for copies by timeout_s of wall time; one that gives up sets *err = 4 (the
// sweep's results are then invalid).  pdl: programmatic dependent launch.
bool fused_config_valid(int L, int tile_z, int depth);
cudaError_t launch_sweeps_fused(uint32_t **cur, uint32_t **nxt, int L, int R, uint64_t seed, int rule, int64_t t0,
                                int64_t n_mcs, int cycle, int tile_z, int depth, int *err, double timeout_s,
                                cudaStream_t s, int64_t *launches, bool pdl = true);

// n_mcs sweeps from completed-sweep count t0; returns the number of launches through
// *launches.
// cycle 0: red then blue every sweep; cycle 1: mixed cycle (random first sublattice per
// sweep and replica, see mixed_first).
cudaError_t launch_sweeps_packed(uint32_t *lat, int L, int R, uint64_t seed, int rule, int64_t t0,
                                 int64_t n_mcs, int cycle, const SweepConfig &cfg, cudaStream_t s,
                                 int64_t *launches);
int mixed_first(uint64_t S, uint32_t t);
// Menger-sponge start of iteration k for every replica (padding words must be zero).
cudaError_t launch_init_menger(uint32_t *lat, int L, int R, uint64_t seed, int k, cudaStream_t s);

// Double-checkerboard update (Supp. Methods I A): blocks of bx*by*bz sites, red blocks
// (block indices summing to an even number) then blue ones; inside a block the sites of one
// parity, then the other.  A block row is the block's x-range of one row (y,z) of one
// sublattice: m words, plus one halo word on each side when the block does not span x.
struct DcbGeom {
    int bx, by, bz;     // block sides in sites
    int nbx, nby, nbz;  // blocks per axis (each even, or 1)
    int m;              // words per block row and sublattice
    int xh;             // 1: block rows carry x-halo words (bx < L)
    int v;              // words per thread: 4 when m is a multiple of 4, else 1
    int off, rs;        // offset of the block's own words and stride of a row in shared memory
    int64_t nblk;       // blocks in the lattice
};
// Fill *d for an L^3 packed lattice (bx = 0: L; by = 0: 16, bz = 0: 8; both L when L <= 16).  False
// when the tiling is not a double checkerboard the kernel supports: bx must be L or a
// multiple of 64 with an even number of blocks, by and bz divisors of L with an even
// quotient (or L), and a block with its halo must fit in 227 KB of shared memory.
bool make_dcb_geom(int L, int bx, int by, int bz, DcbGeom *d);
size_t dcb_smem_bytes(const DcbGeom &d);
// n_mcs double-checkerboard sweeps from t0.  cycle 0: red blocks first, odd sites first in
// every block; cycle 1: colour order per sweep and replica from mixed_first, fine order per
// block from Philox phase 6.
cudaError_t launch_sweeps_dcb(uint32_t *lat, int L, int R, uint64_t seed, int rule, int64_t t0, int64_t n_mcs,
                              int cycle, const DcbGeom &d, cudaStream_t s, int64_t *launches);

// Radially averaged 3-d correlation and structure factor of one lattice (lat_r: replica's
// packed store) through cuFFT; precision 0: single, 1: double.
// out (device): [C(0..nb-1), S(0..nb-1), l]; cnt (device): [n_b (nb), inexact lags].
// Allocates, stream-ordered, radial_scratch_bytes(L, precision) plus cuFFT's work area at the
// first call and keeps them in *p (radial_release frees them).  On a cuFFT failure returns
// cudaErrorUnknown with the cuFFT status in *cufft_status.
struct RadialPlans;
RadialPlans *radial_plans_create();
void radial_release(RadialPlans *p, cudaStream_t s);
void radial_plans_destroy(RadialPlans *p, cudaStream_t s);
int64_t radial_nbins(int L);
size_t radial_scratch_bytes(int L, int precision);
cudaError_t launch_radial(RadialPlans *p, const uint32_t *lat_r, int L, int precision, double c, double *out,
                          int64_t *cnt, cudaStream_t s, int64_t *launches, int *cufft_status);

// ---- plain form: one byte per spin, replica r at plain + r*N. --------------------
cudaError_t launch_init_plain(int8_t *plain, int L, int R, uint64_t seed, cudaStream_t s);
cudaError_t launch_sweeps_plain(int8_t *plain, int L, int R, uint64_t seed, int rule, int64_t t0,
                                int64_t n_mcs, int cycle, cudaStream_t s, int64_t *launches);
// plain -> packed (for the shared measurement kernels) and back.
cudaError_t launch_pack(const int8_t *plain, uint32_t *lat, int L, int R, cudaStream_t s);
cudaError_t launch_unpack(const uint32_t *lat, int8_t *plain, int L, int R, cudaStream_t s);

// ---- measurement on the packed store ----------------------------------------------
// rec: R records of 3 + 3*(L/2+1) int64 (must not alias lat).  Writes t, M, B and the
// correlation sums D_a(r) by the chosen method (CORR_NONE writes D_a(r) = -1).
// CORR_TENSOR needs corr_mma_supported(L), xt_scratch of corr_mma_scratch_bytes(L, R) bytes
// and err (a device int set to 1 if a bounded wait of the tensor-core kernel gave up; the
// records are then incomplete).
enum CorrMethod : int { CORR_NONE = 0, CORR_POPCOUNT = 1, CORR_TENSOR = 2 };
// wait_timeout_s bounds each device-side wait of the tensor-core path (wall time);
// inject_stall (tests) makes one of its CTAs skip a load so that a wait runs out.
cudaError_t launch_measure(const uint32_t *lat, int L, int R, int64_t t, int corr, int64_t *rec,
                           cudaStream_t s, int64_t *launches, uint32_t *xt_scratch = nullptr, int *err = nullptr,
                           double wait_timeout_s = 2.0, int inject_stall = 0);
bool corr_mma_supported(int L);
size_t corr_mma_scratch_bytes(int L, int R);
cudaError_t launch_corr_mma(const uint32_t *lat, int L, int R, int64_t *rec, uint32_t *xt_scratch, int *err,
                            cudaStream_t s, int64_t *launches, double timeout_s, int inject);
// derived: R x [e, m, l_E, l_C]
cudaError_t launch_derived(const int64_t *rec, int L, int R, double c, bool connected, double *derived,
                           cudaStream_t s, int64_t *launches);

}  // namespace ising
