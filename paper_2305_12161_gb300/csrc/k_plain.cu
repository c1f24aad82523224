// Plain form: one signed byte per spin (+1 / -1), site (x,y,z) at x + L*(y + L*z), one
// kernel launch per lattice and half-sweep.  It is the comparison form for the packed
// store: same rule (Eq. 6 at T -> 0), same checkerboard order, same random bits, so the
// trajectories are identical.
//
// A warp handles the 32 sites of one packed storage word (consecutive k of one row of
// sublattice q, x = 2k + p): lane b owns site k = 32*kw + b (or b < L/2 for L < 64).
// Byte loads of a warp span 64 consecutive bytes of a row; the warp's random word is one
// Philox call shared by its lanes.
#include "common.cuh"
#include "kernels.h"

namespace ising {

struct SiteOfLane {
    bool valid;
    int x, y, z, p;
};

__device__ __forceinline__ SiteOfLane site_of_lane(const Geom &g, int64_t sw, int q, int b)
{
    SiteOfLane s;
    const int64_t row = sw / g.W;
    const int kw = (int)(sw - row * g.W);
    s.y = (int)(row % g.L);
    s.z = (int)(row / g.L);
    s.p = (s.y + s.z + q) & 1;
    s.valid = b < g.RB;
    s.x = 2 * (32 * kw + b) + s.p;
    return s;
}

__device__ __forceinline__ int64_t idx(int L, int x, int y, int z)
{
    return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);
}

__global__ void k_init_plain(int8_t *P, Geom g, uint64_t seed)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t N = (int64_t)g.L * g.L * g.L;
    for (int64_t task = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); task < 2 * g.nw;
         task += nwarps) {
        const int q = (int)(task / g.nw);
        const int64_t sw = task - (int64_t)q * g.nw;
        const int r = blockIdx.y;
        const uint32_t rnd = rng_word(g, sw, 0u, (uint32_t)(2 + q), seed + (uint64_t)r);
        const SiteOfLane s = site_of_lane(g, sw, q, lane);
        if (s.valid) P[(int64_t)r * N + idx(g.L, s.x, s.y, s.z)] = ((rnd >> lane) & 1u) ? 1 : -1;
    }
}

template <int RULE>
__global__ void k_sweep_plain(int8_t *P, Geom g, int q, uint32_t t, uint64_t S)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int L = g.L;
    for (int64_t sw = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); sw < g.nw; sw += nwarps) {
        const SiteOfLane s = site_of_lane(g, sw, q, lane);
        int u = 0;
        int8_t old = 0;
        if (s.valid) {
            const int xm = s.x == 0 ? L - 1 : s.x - 1, xp = s.x == L - 1 ? 0 : s.x + 1;
            const int ym = s.y == 0 ? L - 1 : s.y - 1, yp = s.y == L - 1 ? 0 : s.y + 1;
            const int zm = s.z == 0 ? L - 1 : s.z - 1, zp = s.z == L - 1 ? 0 : s.z + 1;
            u = (P[idx(L, xm, s.y, s.z)] > 0) + (P[idx(L, xp, s.y, s.z)] > 0) + (P[idx(L, s.x, ym, s.z)] > 0) +
                (P[idx(L, s.x, yp, s.z)] > 0) + (P[idx(L, s.x, s.y, zm)] > 0) + (P[idx(L, s.x, s.y, zp)] > 0);
            old = P[idx(L, s.x, s.y, s.z)];
        }
        const unsigned ties = __ballot_sync(0xffffffffu, s.valid && u == 3);
        uint32_t rnd = 0u;
        if (RULE == TIE_GLAUBER && ties != 0u) rnd = rng_word(g, sw, t, (uint32_t)q, S);
        if (s.valid) {
            int8_t nw;
            if (u >= 4)
                nw = 1;
            else if (u <= 2)
                nw = -1;
            else if (RULE == TIE_ALWAYS)
                nw = (int8_t)-old;
            else if (RULE == TIE_NEVER)
                nw = old;
            else
                nw = ((rnd >> lane) & 1u) ? (int8_t)-old : old;
            if (nw != old) P[idx(L, s.x, s.y, s.z)] = nw;
        }
    }
}

cudaError_t launch_init_plain(int8_t *plain, int L, int R, uint64_t seed, cudaStream_t s)
{
    const Geom g = make_geom(L);
    const int64_t warps = 2 * g.nw;
    int64_t blocks = (warps + 7) / 8;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    k_init_plain<<<dim3((unsigned)blocks, (unsigned)R), 256, 0, s>>>(plain, g, seed);
    return cudaGetLastError();
}

template <int RULE>
static void sweeps_plain_rule(int8_t *plain, const Geom &g, int R, uint64_t seed, int64_t t0, int64_t n, int cycle,
                              cudaStream_t s, int64_t *launches)
{
    const int64_t N = (int64_t)g.L * g.L * g.L;
    int64_t blocks = (g.nw + 7) / 8;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        for (int h = 0; h < 2; ++h)
            for (int r = 0; r < R; ++r) {  // one launch per lattice
                const uint64_t S = seed + (uint64_t)r;
                const int q = cycle ? (mixed_first(S, t) ^ h) : h;
                k_sweep_plain<RULE><<<(unsigned)blocks, 256, 0, s>>>(plain + (int64_t)r * N, g, q, t, S);
            }
    }
    if (launches) *launches += 2 * n * R;
}

cudaError_t launch_sweeps_plain(int8_t *plain, int L, int R, uint64_t seed, int rule, int64_t t0, int64_t n,
                                int cycle, cudaStream_t s, int64_t *launches)
{
    if (n <= 0) return cudaSuccess;
    const Geom g = make_geom(L);
    switch (rule) {
    case TIE_GLAUBER: sweeps_plain_rule<TIE_GLAUBER>(plain, g, R, seed, t0, n, cycle, s, launches); break;
    case TIE_ALWAYS: sweeps_plain_rule<TIE_ALWAYS>(plain, g, R, seed, t0, n, cycle, s, launches); break;
    default: sweeps_plain_rule<TIE_NEVER>(plain, g, R, seed, t0, n, cycle, s, launches); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Conversions between the byte-per-spin layout and the packed store (bit = 1 for up).
__global__ void k_pack(const int8_t *P, uint32_t *lat, Geom g)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int r = blockIdx.y;
    for (int64_t task = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); task < 2 * g.nw;
         task += nwarps) {
        const int q = (int)(task / g.nw);
        const int64_t sw = task - (int64_t)q * g.nw;
        const SiteOfLane s = site_of_lane(g, sw, q, lane);
        const bool up = s.valid && P[(int64_t)r * N + idx(g.L, s.x, s.y, s.z)] > 0;
        const unsigned word = __ballot_sync(0xffffffffu, up);
        if (lane == 0) lat[(2 * (int64_t)r + q) * g.nw + sw] = word;
    }
}

__global__ void k_unpack(const uint32_t *lat, int8_t *P, Geom g)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t N = (int64_t)g.L * g.L * g.L;
    const int r = blockIdx.y;
    for (int64_t task = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); task < 2 * g.nw;
         task += nwarps) {
        const int q = (int)(task / g.nw);
        const int64_t sw = task - (int64_t)q * g.nw;
        const SiteOfLane s = site_of_lane(g, sw, q, lane);
        const uint32_t word = lat[(2 * (int64_t)r + q) * g.nw + sw];
        if (s.valid) P[(int64_t)r * N + idx(g.L, s.x, s.y, s.z)] = ((word >> lane) & 1u) ? 1 : -1;
    }
}

cudaError_t launch_pack(const int8_t *plain, uint32_t *lat, int L, int R, cudaStream_t s)
{
    const Geom g = make_geom(L);
    int64_t blocks = (2 * g.nw + 7) / 8;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    k_pack<<<dim3((unsigned)blocks, (unsigned)R), 256, 0, s>>>(plain, lat, g);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t *lat, int8_t *plain, int L, int R, cudaStream_t s)
{
    const Geom g = make_geom(L);
    int64_t blocks = (2 * g.nw + 7) / 8;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    k_unpack<<<dim3((unsigned)blocks, (unsigned)R), 256, 0, s>>>(lat, plain, g);
    return cudaGetLastError();
}

}  // namespace ising
