// Plain form: one signed byte per spin (+1 / -1), site (x,y,z) at x + L*(y + L*z), one
// kernel launch per lattice and half-sweep.  It is the comparison form for the packed
// store: same rule (Eq. 6 at T -> 0), same checkerboard order, same random bits, so the
// trajectories are identical.
//
// A warp handles the 32 sites of one packed storage word (consecutive k of one row of
// sublattice q, x = 2k + p): lane b owns site k = 32*kw + b (or b < L/2 for L < 64).
// Byte loads of a warp span 64 consecutive bytes of a row; the warp's random word is one
// Philox call shared by its lanes.
#include <algorithm>

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

// Half-sweep of the plain form with CH chunks of 16 sites per thread (L a multiple of 16 CH).
// A thread owns the 16 CH bytes x0 .. x0 + 16 CH - 1 (x0 = 16 CH cp) of row (y, z): 16-byte
// loads of its own bytes and of the same bytes in rows y - 1, y + 1 and planes z - 1, z + 1
// (coalesced across the warp; the neighbour rows are re-read from L2 by the threads that own
// them).  The x edge bytes come from the adjacent lanes by shuffles (a direct byte load at a
// row or warp edge).  All bytes are evaluated four to a 32-bit word: bit 1 of a byte is set
// exactly for a down spin (0xFF; up is 0x01), so d2 = the sum of the six neighbour words
// masked to bit 1 is twice the number of down neighbours per byte (at most 12: no carry
// between bytes); adding 0x7A or 0x78 to a byte sets its bit 7 when d2 >= 6 (u <= 3) or
// d2 >= 8 (u <= 2).  The bytes of sublattice q (every other byte, x0 even) take the new
// value; the others are stored back unchanged, and a chunk is stored only if one of its bytes
// changed.  A site's random bit is bit (h & 31) of word (h >> 5) & 3 of the Philox group
// h >> 7 of its compressed index h = (x >> 1) + (L/2)(y + L z), as for every other kernel:
// the 8 CH sites of sublattice q of a thread are 8 CH consecutive h inside one output word,
// so one draw serves all of them (CH = 2 halves the draws per site).
// a + b on the FMA pipe: a multiply-add by `one`, a run-time 1 the compiler cannot fold, so
// that the adds of the byte counts do not compete with the bitwise work for the ALU pipe
__device__ __forceinline__ uint32_t fma_add(uint32_t a, uint32_t one, uint32_t b)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "r"(b));
    return r;
}

template <int RULE, int CH>
__global__ void __launch_bounds__(256) k_sweep_plain16(int8_t *P, int L, int q, uint32_t t, uint64_t S, uint32_t one)
{
    constexpr uint32_t FULL = 0xffffffffu, M2 = 0x02020202u, B7 = 0x80808080u;
    constexpr int NW = 4 * CH;            // 32-bit words of a thread
    const int W = L >> 4;                 // chunks per row (<= 256)
    const int WP = W / CH;                // threads per row
    const int rpc = 256 / WP;             // rows of a CTA pass
    const int tr = (int)threadIdx.x / WP;  // this thread's row in the pass, and its first chunk
    const int cp = (int)threadIdx.x - tr * WP;
    const int cx0 = CH * cp;
    const int lane = threadIdx.x & 31;
    const int64_t plane = (int64_t)L * L;
    const int z = blockIdx.y;             // one plane per grid row: no division in the loop
    const int64_t dzm = (z == 0 ? L - 1 : -1) * plane, dzp = (z == L - 1 ? 1 - L : 1) * plane;
    // the pass loop is uniform over the CTA, so whole warps meet at the shuffles; threads past
    // the pass's rows (WP not a power of two) or past the plane compute on row L - 1 and store
    // nothing
    for (int yb = blockIdx.x * rpc; yb < L; yb += gridDim.x * rpc) {
        const bool valid = tr < rpc && yb + tr < L;
        const int y = valid ? yb + tr : L - 1;
        const uint32_t row = (uint32_t)z * (uint32_t)L + (uint32_t)y;
        const int64_t base = (int64_t)row * L;  // first byte of the row
        const int64_t o = base + 16 * cx0;
        const int64_t dym = (y == 0 ? L - 1 : -1) * (int64_t)L, dyp = (y == L - 1 ? 1 - L : 1) * (int64_t)L;
        uint32_t w[NW], a[NW], b[NW], e[NW], f[NW];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const uint4 v = *reinterpret_cast<const uint4 *>(P + o + 16 * c);
            const uint4 ym = *reinterpret_cast<const uint4 *>(P + o + 16 * c + dym);
            const uint4 yp = *reinterpret_cast<const uint4 *>(P + o + 16 * c + dyp);
            const uint4 zm = *reinterpret_cast<const uint4 *>(P + o + 16 * c + dzm);
            const uint4 zp = *reinterpret_cast<const uint4 *>(P + o + 16 * c + dzp);
            w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
            a[4 * c] = ym.x; a[4 * c + 1] = ym.y; a[4 * c + 2] = ym.z; a[4 * c + 3] = ym.w;
            b[4 * c] = yp.x; b[4 * c + 1] = yp.y; b[4 * c + 2] = yp.z; b[4 * c + 3] = yp.w;
            e[4 * c] = zm.x; e[4 * c + 1] = zm.y; e[4 * c + 2] = zm.z; e[4 * c + 3] = zm.w;
            f[4 * c] = zp.x; f[4 * c + 1] = zp.y; f[4 * c + 2] = zp.z; f[4 * c + 3] = zp.w;
        }
        // x edges: byte x0 - 1 (top byte of the chunk before) and the byte after the thread's
        // last chunk (low byte of the next); lanes hold consecutive chunk runs of a row
        uint32_t left = __shfl_up_sync(FULL, w[NW - 1], 1);
        uint32_t right = __shfl_down_sync(FULL, w[0], 1);
        if (lane == 0 || cp == 0) left = (uint32_t)(uint8_t)P[base + (cx0 == 0 ? L - 1 : 16 * cx0 - 1)] << 24;
        if (lane == 31 || cp == WP - 1)
            right = (uint32_t)(uint8_t)P[base + (cx0 + CH == W ? 0 : 16 * (cx0 + CH))];
        const int pq = (y + z + q) & 1;  // sublattice-q bytes: j % 2 == pq
        const uint32_t Mq = pq ? 0x80008000u : 0x00800080u;
        uint32_t ge4[NW], tie[NW], old7[NW], anytie = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t xl = __funnelshift_l(k ? w[k - 1] : left, w[k], 8);         // byte j - 1
            const uint32_t xr = __funnelshift_r(w[k], k < NW - 1 ? w[k + 1] : right, 8);  // byte j + 1
            const uint32_t d2 = fma_add(xl & M2, one, fma_add(xr & M2, one, fma_add(a[k] & M2, one,
                                fma_add(b[k] & M2, one, fma_add(e[k] & M2, one, f[k] & M2)))));
            const uint32_t ge3 = fma_add(d2, one, 0x7A7A7A7Au) & B7;
            ge4[k] = fma_add(d2, one, 0x78787878u) & B7;
            tie[k] = ge3 & ~ge4[k] & Mq;
            old7[k] = w[k] & B7;
            anytie |= tie[k];
        }
        uint32_t rnd = 0u;
        if (RULE == TIE_GLAUBER && __ballot_sync(FULL, anytie != 0u)) {
            // every lane draws its own group (the warp issues the rounds once)
            const uint64_t h0 = (uint64_t)(8 * cx0) + (uint64_t)(L / 2) * row;
            const U4 ph = philox4x32_10((uint32_t)(h0 >> 7), t, (uint32_t)q, 0u, (uint32_t)S, (uint32_t)(S >> 32));
            rnd = (pick(ph, (int)((h0 >> 5) & 3)) >> (h0 & 31)) & (CH == 2 ? 0xffffu : 0xffu);
        }
        uint32_t out[NW];
        bool changed[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) changed[c] = false;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            uint32_t tau;
            if (RULE == TIE_GLAUBER) {
                // sites m = 2k, 2k + 1 of the thread sit at bytes pq and 2 + pq of word k
                const uint32_t r2 = (rnd >> (2 * k)) & 3u;
                const uint32_t r7 = ((r2 & 1u) << (7 + 8 * pq)) | ((r2 >> 1) << (23 + 8 * pq));
                tau = old7[k] ^ r7;
            } else if (RULE == TIE_ALWAYS) {
                tau = ~old7[k] & B7;
            } else {
                tau = old7[k];
            }
            const uint32_t nd = (ge4[k] & Mq) | (tie[k] & tau) | (old7[k] & ~Mq);  // new down bits
            out[k] = (nd >> 7) * 0xFEu + 0x01010101u;
            changed[k / 4] |= out[k] != w[k];
        }
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (changed[c] && valid)
                *reinterpret_cast<uint4 *>(P + o + 16 * c) =
                    make_uint4(out[4 * c], out[4 * c + 1], out[4 * c + 2], out[4 * c + 3]);
    }
}

template <int RULE>
static void sweeps_plain_rule(int8_t *plain, const Geom &g, int R, uint64_t seed, int64_t t0, int64_t n, int cycle,
                              cudaStream_t s, int64_t *launches)
{
    const int64_t N = (int64_t)g.L * g.L * g.L;
    int64_t blocks = (g.nw + 7) / 8;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    // 16 or 32 bytes per thread: one grid row per plane, each CTA about eight passes of its
    // 256 threads' rows along y
    const int rpc = g.L >= 16 ? 256 / (g.L / 16) : 1;
    const dim3 grid16((unsigned)std::max(1, (g.L / rpc + 7) / 8), (unsigned)g.L);
    const int rpc2 = g.L >= 32 ? 256 / (g.L / 32) : 1;  // 32 bytes per thread
    const dim3 grid32((unsigned)std::max(1, (g.L / rpc2 + 7) / 8), (unsigned)g.L);
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        for (int h = 0; h < 2; ++h)
            for (int r = 0; r < R; ++r) {  // one launch per lattice
                const uint64_t S = seed + (uint64_t)r;
                const int q = cycle ? (mixed_first(S, t) ^ h) : h;
                if (g.L % 32 == 0)
                    k_sweep_plain16<RULE, 2><<<grid32, 256, 0, s>>>(plain + (int64_t)r * N, g.L, q, t, S, 1u);
                else if (g.L % 16 == 0)
                    k_sweep_plain16<RULE, 1><<<grid16, 256, 0, s>>>(plain + (int64_t)r * N, g.L, q, t, S, 1u);
                else
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
