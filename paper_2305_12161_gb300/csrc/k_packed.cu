// Packed-form kernels: the T = infinity initial state and the checkerboard half-sweep
// (Methods, "Checkerboard update"; acceptance Eq. (6) at T -> 0) on 1-bit sublattices.
//
// Two sweep variants, bit-identical:
//   WORD   — one thread per 32-bit word; neighbours through the read-only cache.  Any
//            supported L (multiples of 64, and 4..32 with one padded word per row).
//   ZMARCH — for L >= 256 (a row is W/4 >= 1 uint4): a CTA owns a tile of TY full
//            rows and marches it through TZ consecutive planes.  Planes of the other
//            sublattice (with one halo row above and below) and of the own sublattice
//            stream into a shared-memory ring through cp.async, two planes ahead, so
//            every word of either array is read from HBM about once per half-sweep.
//            Each thread updates 128 spins (one uint4, one Philox group) per plane.
#include "common.cuh"
#include "kernels.h"

namespace ising {

// ---------------------------------------------------------------------------------
// Initial state: sublattice q of replica r is the Philox output of phase 2+q at t = 0.
__global__ void k_init_packed_wide(uint32_t *lat, Geom g, uint64_t seed)
{
    // L >= 64: storage words coincide with compressed-index words; one Philox call
    // yields the four words of a group.
    const int r = blockIdx.y, q = blockIdx.z;
    uint4 *S4 = reinterpret_cast<uint4 *>(lat + (2 * (int64_t)r + q) * g.nw);
    const uint64_t S = seed + (uint64_t)r;
    const int64_t ng = g.nw >> 2;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < ng;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const U4 o = philox4x32_10((uint32_t)gi, 0u, (uint32_t)(2 + q), 0u, (uint32_t)S, (uint32_t)(S >> 32));
        S4[gi] = make_uint4(o.x, o.y, o.z, o.w);
    }
}

__global__ void k_init_packed_small(uint32_t *lat, Geom g, uint64_t seed)
{
    const int r = blockIdx.y, q = blockIdx.z;
    uint32_t *Sq = lat + (2 * (int64_t)r + q) * g.nw;
    const uint64_t S = seed + (uint64_t)r;
    for (int64_t sw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sw < g.nw;
         sw += (int64_t)gridDim.x * blockDim.x)
        Sq[sw] = rng_word(g, sw, 0u, (uint32_t)(2 + q), S);
}

static int grid_for(int64_t items, int block, int cap)
{
    int64_t b = (items + block - 1) / block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_init_packed(uint32_t *lat, int L, int R, uint64_t seed, cudaStream_t s)
{
    const Geom g = make_geom(L);
    if (L >= 64) {
        dim3 grid(grid_for(g.nw / 4, 256, 65535), R, 2);
        k_init_packed_wide<<<grid, 256, 0, s>>>(lat, g, seed);
    } else {
        dim3 grid(grid_for(g.nw, 256, 65535), R, 2);
        k_init_packed_small<<<grid, 256, 0, s>>>(lat, g, seed);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// WORD variant: one 32-bit word (32 spins of one row) per thread.
template <int RULE>
__global__ void k_sweep_word(uint32_t *lat, Geom g, int q, uint32_t t, uint64_t seed)
{
    const int r = blockIdx.y;
    uint32_t *S = lat + (2 * (int64_t)r + q) * g.nw;
    const uint32_t *O = lat + (2 * (int64_t)r + (1 - q)) * g.nw;
    const uint64_t key = seed + (uint64_t)r;
    for (int64_t sw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sw < g.nw;
         sw += (int64_t)gridDim.x * blockDim.x) {
        const Nbrs n = load_nbrs(O, g, sw, q);
        uint32_t ge4, eq3;
        count6(n.C, n.X, n.Ym, n.Yp, n.Zm, n.Zp, ge4, eq3);
        const uint32_t s = S[sw];
        uint32_t rnd = 0u;
        if (RULE == TIE_GLAUBER && eq3 != 0u) rnd = rng_word(g, sw, t, (uint32_t)q, key);
        S[sw] = resolve<RULE>(s, ge4, eq3, rnd);
    }
}

// ---------------------------------------------------------------------------------
// ZMARCH variant.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int ZM_AHEAD = 2;            // copy groups in flight beyond the one consumed
constexpr int ZM_NSO = 3 + ZM_AHEAD;   // ring slots for other-sublattice planes
constexpr int ZM_NSQ = 1 + ZM_AHEAD;   // ring slots for own-sublattice planes

static size_t zmarch_smem_bytes(int L, int TY)
{
    const int W4 = L / 256;
    return sizeof(uint4) * (size_t)(ZM_NSO * (TY + 2) * W4 + ZM_NSQ * TY * W4);
}

// Copy group gi (gi = 0, 1, ...) of a tile holds the other sublattice's plane
// z0 - 1 + gi (TY + 2 rows: the tile and one halo row on each side) and, for gi >= 2,
// the own sublattice's plane z0 + gi - 2.  Step i (plane z = z0 + i) needs the other
// planes z-1, z, z+1 (groups i, i+1, i+2) and own plane z (group i+2).
template <int RULE>
__global__ void __launch_bounds__(1024) k_sweep_zmarch(uint32_t *lat, Geom g, int q, uint32_t t,
                                                       uint64_t seed, int TY, int TZ)
{
    extern __shared__ uint4 zsm[];
    const int L = g.L;
    const int W4 = g.W >> 2;
    const int NT = blockDim.x;  // TY * W4
    const int tid = threadIdx.x;
    const int ty = tid / W4, cx = tid - ty * W4;
    const int nty = L / TY;
    const int y0 = (int)(blockIdx.x % nty) * TY;
    const int z0 = (int)(blockIdx.x / nty) * TZ;
    const int r = blockIdx.y;
    uint4 *S4 = reinterpret_cast<uint4 *>(lat + (2 * (int64_t)r + q) * g.nw);
    const uint4 *O4 = reinterpret_cast<const uint4 *>(lat + (2 * (int64_t)r + (1 - q)) * g.nw);
    const uint64_t key = seed + (uint64_t)r;
    const int OSZ = (TY + 2) * W4;
    const int QSZ = TY * W4;
    uint4 *osm = zsm;
    uint4 *qsm = zsm + ZM_NSO * OSZ;
    const int64_t plane4 = (int64_t)L * W4;

    auto issue = [&](int gi) {
        if (gi <= TZ + 1) {
            int pz = z0 - 1 + gi;
            pz = pz < 0 ? pz + L : (pz >= L ? pz - L : pz);
            uint4 *dst = osm + (gi % ZM_NSO) * OSZ;
            const uint4 *src = O4 + (int64_t)pz * plane4;
            for (int e = tid; e < OSZ; e += NT) {
                const int ry = e / W4, ex = e - ry * W4;
                int yy = y0 - 1 + ry;
                yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
                cp_async16(dst + e, src + (int64_t)yy * W4 + ex);
            }
        }
        if (gi >= 2 && gi <= TZ + 1) {
            const int pz = z0 + gi - 2;
            cp_async16(qsm + (gi % ZM_NSQ) * QSZ + tid, S4 + (int64_t)pz * plane4 + (int64_t)(y0 + ty) * W4 + cx);
        }
        cp_async_commit();
    };

#pragma unroll 1
    for (int gi = 0; gi < ZM_AHEAD + 2; ++gi) issue(gi);

    const int y = y0 + ty;
    const int cxl = cx == 0 ? W4 - 1 : cx - 1;
    const int cxr = cx == W4 - 1 ? 0 : cx + 1;
#pragma unroll 1
    for (int i = 0; i < TZ; ++i) {
        cp_async_wait<ZM_AHEAD - 1>();
        __syncthreads();
        issue(i + 2 + ZM_AHEAD);  // refills the slots read in step i-1 only

        const int z = z0 + i;
        const uint4 *Oz = osm + ((i + 1) % ZM_NSO) * OSZ;
        const uint4 c = Oz[(ty + 1) * W4 + cx];
        const uint4 ym = Oz[ty * W4 + cx];
        const uint4 yp = Oz[(ty + 2) * W4 + cx];
        const uint4 zm = osm[(i % ZM_NSO) * OSZ + (ty + 1) * W4 + cx];
        const uint4 zp = osm[((i + 2) % ZM_NSO) * OSZ + (ty + 1) * W4 + cx];
        const uint4 s = qsm[((i + 2) % ZM_NSQ) * QSZ + tid];
        const int p = (y + z + q) & 1;
        uint4 X;
        if (p == 0) {  // x-1 neighbour: bit k-1, carried in from the word on the left
            const uint32_t e = Oz[(ty + 1) * W4 + cxl].w;
            X.x = __funnelshift_l(e, c.x, 1);
            X.y = __funnelshift_l(c.x, c.y, 1);
            X.z = __funnelshift_l(c.y, c.z, 1);
            X.w = __funnelshift_l(c.z, c.w, 1);
        } else {       // x+1 neighbour: bit k+1, carried in from the word on the right
            const uint32_t e = Oz[(ty + 1) * W4 + cxr].x;
            X.x = __funnelshift_r(c.x, c.y, 1);
            X.y = __funnelshift_r(c.y, c.z, 1);
            X.z = __funnelshift_r(c.z, c.w, 1);
            X.w = __funnelshift_r(c.w, e, 1);
        }
        uint32_t g0, g1, g2, g3, e0, e1, e2, e3;
        count6(c.x, X.x, ym.x, yp.x, zm.x, zp.x, g0, e0);
        count6(c.y, X.y, ym.y, yp.y, zm.y, zp.y, g1, e1);
        count6(c.z, X.z, ym.z, yp.z, zm.z, zp.z, g2, e2);
        count6(c.w, X.w, ym.w, yp.w, zm.w, zp.w, g3, e3);
        const int64_t gidx = ((int64_t)z * L + y) * W4 + cx;  // Philox group = word >> 2
        U4 o{0u, 0u, 0u, 0u};
        if (RULE == TIE_GLAUBER && (e0 | e1 | e2 | e3) != 0u)
            o = philox4x32_10((uint32_t)gidx, t, (uint32_t)q, 0u, (uint32_t)key, (uint32_t)(key >> 32));
        uint4 nw;
        nw.x = resolve<RULE>(s.x, g0, e0, o.x);
        nw.y = resolve<RULE>(s.y, g1, e1, o.y);
        nw.z = resolve<RULE>(s.z, g2, e2, o.z);
        nw.w = resolve<RULE>(s.w, g3, e3, o.w);
        S4[gidx] = nw;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------
// ZFAST variant: the z-marching scheme specialised on the row width W4 (uint4 per row)
// with 256 threads, so a tile is TY = 256 / W4 full rows and all index arithmetic is
// compile-time.  Per plane each thread reads one new other-sublattice word of its own
// column (z+1) and keeps z-1 and z in registers; the y-neighbours and the x edge come
// from the shared ring; its own-sublattice word is prefetched from global memory two
// planes ahead into registers.  Philox round keys are computed once per thread.  The rows
// a warp computes share their parity, so the direction of the x-neighbour shift (which
// alternates with y + z) is the same for the whole warp; own-word pointer and Philox
// counter advance by one plane per step.
template <int RULE, int W4>
__global__ void __launch_bounds__(256) k_sweep_zfast(uint32_t *lat, Geom g, int q, uint32_t t, uint64_t seed, int TZ)
{
    constexpr int NT = 256, TY = NT / W4;
    constexpr int OSZ = (TY + 2) * W4;  // uint4 per ring slot: the tile and one halo row each side
    constexpr int NS = 5;               // slots: planes z, z+1 being read, z+2, z+3 in flight, 1 spare
    constexpr int RW = 32 / W4;         // rows per warp
    __shared__ uint4 ring[NS * OSZ];
    pdl_enter();
    const int L = g.L;
    const int tid = threadIdx.x;
    const int nty = L / TY;
    const int y0 = (int)(blockIdx.x % nty) * TY;
    const int z0 = (int)(blockIdx.x / nty) * TZ;
    const int r = blockIdx.y;
    uint4 *S4 = reinterpret_cast<uint4 *>(lat + (2 * (int64_t)r + q) * g.nw);
    const uint4 *O4 = reinterpret_cast<const uint4 *>(lat + (2 * (int64_t)r + (1 - q)) * g.nw);
    const PhiloxKeys keys = philox_keys(seed + (uint64_t)r);
    const int64_t plane4 = (int64_t)L * W4;

    // copies: thread tid fills ring row tid / W4 (global row y0-1+tid/W4) and, for
    // tid < 2*W4, ring row TY + tid/W4
    const int ly = tid / W4, lx = tid % W4;
    int ya = y0 - 1 + ly;
    ya = ya < 0 ? ya + L : ya;
    const int64_t offa = (int64_t)ya * W4 + lx;
    const bool halo = tid < 2 * W4;
    int yb = y0 - 1 + TY + ly;  // ly is 0 or 1 here
    yb = yb >= L ? yb - L : yb;
    const int64_t offb = (int64_t)yb * W4 + lx;

    // compute: the rows of a warp share their parity, so the x-neighbour direction (which
    // alternates with y + z) is uniform across the warp
    const int warp = tid >> 5, lane = tid & 31;
    const int cx = lane % W4;
    const int ty = (warp >> 1) * 2 * RW + (warp & 1) + 2 * (lane / W4);
    const int y = y0 + ty;
    const int64_t own = (int64_t)y * W4 + cx;  // own column within a plane

    auto issue = [&](int gi) {  // other-sublattice plane z0-1+gi into slot gi % NS
        if (gi <= TZ + 1) {
            int pz = z0 - 1 + gi;
            pz = pz < 0 ? pz + L : (pz >= L ? pz - L : pz);
            const uint4 *src = O4 + (int64_t)pz * plane4;
            uint4 *dst = ring + (gi % NS) * OSZ;
            cp_async16(dst + tid, src + offa);
            if (halo) cp_async16(dst + NT + tid, src + offb);
        }
        cp_async_commit();
    };

#pragma unroll 1
    for (int gi = 0; gi < 4; ++gi) issue(gi);
    uint4 *sp = S4 + (int64_t)z0 * plane4 + own;  // own word at plane z
    uint4 sA = sp[0];
    uint4 sB = TZ > 1 ? sp[plane4] : sA;
    cp_async_wait<2>();  // groups 0 and 1 (planes z0-1, z0) have landed
    __syncthreads();
    uint4 cm = ring[0 * OSZ + (ty + 1) * W4 + cx];  // plane z-1, own column
    uint4 cc = ring[1 * OSZ + (ty + 1) * W4 + cx];  // plane z
    const int cxl = (cx + W4 - 1) % W4, cxr = (cx + 1) % W4;
    int sz = 1;  // slot of plane z
    int p = (y + z0 + q) & 1;
    uint32_t gidx = (uint32_t)((int64_t)z0 * plane4 + own);  // Philox group = word >> 2
    const uint32_t gstep = (uint32_t)plane4;
#pragma unroll 1  // unrolling by two measured 5% slower
    for (int i = 0; i < TZ; ++i) {
        cp_async_wait<1>();  // group i+2 (plane z+1) has landed
        __syncthreads();
        issue(i + 4);        // overwrites the slot of plane z-2, last read in step i-1
        const int szp = sz == NS - 1 ? 0 : sz + 1;
        const uint4 *Oz = ring + sz * OSZ;
        const uint4 cp = ring[szp * OSZ + (ty + 1) * W4 + cx];
        const uint4 ym = Oz[ty * W4 + cx];
        const uint4 yp = Oz[(ty + 2) * W4 + cx];
        const uint4 s = sA;
        sA = sB;
        if (i + 2 < TZ) sB = sp[2 * plane4];
        uint4 X;
        if (p == 0) {
            const uint32_t e = Oz[(ty + 1) * W4 + cxl].w;
            X.x = __funnelshift_l(e, cc.x, 1);
            X.y = __funnelshift_l(cc.x, cc.y, 1);
            X.z = __funnelshift_l(cc.y, cc.z, 1);
            X.w = __funnelshift_l(cc.z, cc.w, 1);
        } else {
            const uint32_t e = Oz[(ty + 1) * W4 + cxr].x;
            X.x = __funnelshift_r(cc.x, cc.y, 1);
            X.y = __funnelshift_r(cc.y, cc.z, 1);
            X.z = __funnelshift_r(cc.z, cc.w, 1);
            X.w = __funnelshift_r(cc.w, e, 1);
        }
        *sp = new_spins4<RULE>(s, cc, X, ym, yp, cm, cp, gidx, t, (uint32_t)q, keys);
        sp += plane4;
        gidx += gstep;
        p ^= 1;
        cm = cc;
        cc = cp;
        sz = szp;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------
// ZDEEP variant: the ZFAST tile walk with a deeper copy pipeline.  Both sublattices'
// planes stream through shared-memory rings by cp.async, AHEAD planes beyond the one
// being consumed (other ring AHEAD+3 slots, own ring AHEAD+1), and the Philox round keys
// are recomputed per call instead of held in registers, so more CTAs fit per SM.  The
// sweep is bound by memory latency (its speed does not change between dense-tie and
// sparse-tie times), which both measures address: more bytes in flight per SM.
template <int RULE, int W4, int AHEAD>
__global__ void __launch_bounds__(256) k_sweep_zdeep(uint32_t *lat, Geom g, int q, uint32_t t, uint64_t seed, int TZ)
{
    constexpr int NT = 256, TY = NT / W4;
    constexpr int OSZ = (TY + 2) * W4;
    constexpr int NS = AHEAD + 3, NQ = AHEAD + 1;
    extern __shared__ uint4 dsm[];
    uint4 *ring = dsm;             // NS * OSZ
    uint4 *qring = dsm + NS * OSZ; // NQ * NT
    const int L = g.L;
    const int tid = threadIdx.x;
    const int ty = tid / W4, cx = tid % W4;
    const int nty = L / TY;
    const int y0 = (int)(blockIdx.x % nty) * TY;
    const int z0 = (int)(blockIdx.x / nty) * TZ;
    const int r = blockIdx.y;
    uint4 *S4 = reinterpret_cast<uint4 *>(lat + (2 * (int64_t)r + q) * g.nw);
    const uint4 *O4 = reinterpret_cast<const uint4 *>(lat + (2 * (int64_t)r + (1 - q)) * g.nw);
    const uint64_t key = seed + (uint64_t)r;
    const int64_t plane4 = (int64_t)L * W4;
    int ya = y0 - 1 + ty;
    ya = ya < 0 ? ya + L : ya;
    const int64_t offa = (int64_t)ya * W4 + cx;
    const bool halo = tid < 2 * W4;
    int yb = y0 - 1 + TY + ty;
    yb = yb >= L ? yb - L : yb;
    const int64_t offb = (int64_t)yb * W4 + cx;
    const int y = y0 + ty;
    const int64_t own = (int64_t)y * W4 + cx;

    // group gi: other plane z0-1+gi -> ring slot gi % NS; own plane z0+gi-2 (gi >= 2) ->
    // qring slot gi % NQ.  Slots are tracked incrementally.
    int so_issue = 0, sq_issue = 0;
    auto issue = [&](int gi) {
        if (gi <= TZ + 1) {
            int pz = z0 - 1 + gi;
            pz = pz < 0 ? pz + L : (pz >= L ? pz - L : pz);
            const uint4 *src = O4 + (int64_t)pz * plane4;
            uint4 *dst = ring + so_issue * OSZ;
            cp_async16(dst + tid, src + offa);
            if (halo) cp_async16(dst + NT + tid, src + offb);
        }
        if (gi >= 2 && gi <= TZ + 1) cp_async16(qring + sq_issue * NT + tid, S4 + (int64_t)(z0 + gi - 2) * plane4 + own);
        cp_async_commit();
        so_issue = so_issue == NS - 1 ? 0 : so_issue + 1;
        sq_issue = sq_issue == NQ - 1 ? 0 : sq_issue + 1;
    };

#pragma unroll 1
    for (int gi = 0; gi < AHEAD + 2; ++gi) issue(gi);
    cp_async_wait<AHEAD>();  // groups 0 and 1 have landed
    __syncthreads();
    uint4 cm = ring[0 * OSZ + (ty + 1) * W4 + cx];
    uint4 cc = ring[1 * OSZ + (ty + 1) * W4 + cx];
    const int cxl = (cx + W4 - 1) % W4, cxr = (cx + 1) % W4;
    int sz = 1;       // ring slot of other plane z  (group i+1)
    int sqz = 2 % NQ; // qring slot of own plane z   (group i+2)
#pragma unroll 1
    for (int i = 0; i < TZ; ++i) {
        cp_async_wait<AHEAD - 1>();  // group i+2 has landed
        __syncthreads();
        issue(i + 2 + AHEAD);        // overwrites other plane z-2 and own plane z-1 (both done)
        const int z = z0 + i;
        const int szp = sz == NS - 1 ? 0 : sz + 1;
        const uint4 *Oz = ring + sz * OSZ;
        const uint4 cp = ring[szp * OSZ + (ty + 1) * W4 + cx];
        const uint4 ym = Oz[ty * W4 + cx];
        const uint4 yp = Oz[(ty + 2) * W4 + cx];
        const uint4 s = qring[sqz * NT + tid];
        const int p = (y + z + q) & 1;
        uint4 X;
        if (p == 0) {
            const uint32_t e = Oz[(ty + 1) * W4 + cxl].w;
            X.x = __funnelshift_l(e, cc.x, 1);
            X.y = __funnelshift_l(cc.x, cc.y, 1);
            X.z = __funnelshift_l(cc.y, cc.z, 1);
            X.w = __funnelshift_l(cc.z, cc.w, 1);
        } else {
            const uint32_t e = Oz[(ty + 1) * W4 + cxr].x;
            X.x = __funnelshift_r(cc.x, cc.y, 1);
            X.y = __funnelshift_r(cc.y, cc.z, 1);
            X.z = __funnelshift_r(cc.z, cc.w, 1);
            X.w = __funnelshift_r(cc.w, e, 1);
        }
        uint32_t g0, g1, g2, g3, e0, e1, e2, e3;
        count6(cc.x, X.x, ym.x, yp.x, cm.x, cp.x, g0, e0);
        count6(cc.y, X.y, ym.y, yp.y, cm.y, cp.y, g1, e1);
        count6(cc.z, X.z, ym.z, yp.z, cm.z, cp.z, g2, e2);
        count6(cc.w, X.w, ym.w, yp.w, cm.w, cp.w, g3, e3);
        const uint32_t gidx = (uint32_t)((int64_t)z * plane4 + own);
        U4 o{0u, 0u, 0u, 0u};
        if (RULE == TIE_GLAUBER && (e0 | e1 | e2 | e3) != 0u)
            o = philox4x32_10(gidx, t, (uint32_t)q, 0u, (uint32_t)key, (uint32_t)(key >> 32));
        uint4 nw;
        nw.x = resolve<RULE>(s.x, g0, e0, o.x);
        nw.y = resolve<RULE>(s.y, g1, e1, o.y);
        nw.z = resolve<RULE>(s.z, g2, e2, o.z);
        nw.w = resolve<RULE>(s.w, g3, e3, o.w);
        S4[(int64_t)z * plane4 + own] = nw;
        cm = cc;
        cc = cp;
        sz = szp;
        sqz = sqz == NQ - 1 ? 0 : sqz + 1;
    }
    cp_async_wait<0>();
}

static size_t zdeep_smem_bytes(int L, int ahead)
{
    const int W4 = L / 256, TY = 256 / W4;
    return sizeof(uint4) * (size_t)((ahead + 3) * (TY + 2) * W4 + (ahead + 1) * 256);
}

// ---------------------------------------------------------------------------------
static bool zfast_width_ok(int L) { return L % 256 == 0 && (L / 256 == 1 || L / 256 == 2 || L / 256 == 4 || L / 256 == 8); }

bool sweep_config_valid(int L, const SweepConfig &c)
{
    if (c.variant == VARIANT_WORD) return true;
    if (c.variant == VARIANT_ZFUSE) return fused_config_valid(L, c.tile_z, c.depth);
    if (c.variant == VARIANT_ZFAST)
        return L >= 256 && zfast_width_ok(L) && c.tile_z >= 1 && L % c.tile_z == 0 && L % (256 / (L / 256)) == 0;
    if (c.variant == VARIANT_ZDEEP)
        return L >= 256 && zfast_width_ok(L) && c.tile_z >= 1 && L % c.tile_z == 0 && L % (256 / (L / 256)) == 0 &&
               c.depth >= 2 && c.depth <= 4;
    if (c.variant != VARIANT_ZMARCH) return false;
    if (L < 256 || L % 256 != 0) return false;
    const int W4 = L / 256;
    if (c.tile_y < 1 || c.tile_z < 1 || L % c.tile_y != 0 || L % c.tile_z != 0) return false;
    if (c.tile_y * W4 > 1024 || c.tile_y * W4 < 32) return false;
    if (zmarch_smem_bytes(L, c.tile_y) > 200 * 1024) return false;
    return true;
}

SweepConfig default_sweep_config(int L, int R)
{
    SweepConfig c{VARIANT_WORD, 0, 0, 0};
    if (L >= 256 && L % 256 == 0) {
        const int W4 = L / 256;
        int ty = 256 / W4;
        if (ty < 8) ty = 8;
        while (ty > 1 && (L % ty != 0 || ty * W4 > 1024)) ty >>= 1;
        int tz = 32;
        while (tz > 1 && L % tz != 0) tz >>= 1;
        // keep at least ~4 CTAs per SM-worth of tiles on small lattices
        while (tz > 4 && (int64_t)(L / ty) * (L / tz) * R < 4 * device_sms()) tz >>= 1;
        c = SweepConfig{VARIANT_ZMARCH, ty, tz, 0};
        if (!sweep_config_valid(L, c)) c = SweepConfig{VARIANT_WORD, 0, 0, 0};
        if (zfast_width_ok(L)) {
            const int fty = 256 / W4;
            int ftz = 32;
            while (ftz > 4 && (int64_t)(L / fty) * (L / ftz) * R < 4 * device_sms()) ftz >>= 1;
            const SweepConfig f{VARIANT_ZFAST, fty, ftz, 2};
            if (sweep_config_valid(L, f)) c = f;
        }
    }
    return c;
}

// One half-sweep of sublattice q at sweep t for R replicas starting at `lat` (replica r
// keyed seed + r), with the configured kernel variant.
template <int RULE>
static cudaError_t half_sweep_rule(uint32_t *lat, int L, int R, uint64_t seed, int q, uint32_t t,
                                   const SweepConfig &cfg, cudaStream_t s)
{
    const Geom g = make_geom(L);
    if (cfg.variant == VARIANT_ZFUSE) return cudaErrorInvalidValue;  // needs two stores: launch_sweeps_fused
    if (cfg.variant == VARIANT_ZDEEP) {
        const int W4 = L / 256;
        const dim3 grid((unsigned)((L / (256 / W4)) * (L / cfg.tile_z)), (unsigned)R);
        const size_t smem = zdeep_smem_bytes(L, cfg.depth);
        void *fn = nullptr;
#define ZD_CASE(w, a) \
    if (W4 == w && cfg.depth == a) fn = (void *)k_sweep_zdeep<RULE, w, a>;
        ZD_CASE(1, 2) ZD_CASE(1, 3) ZD_CASE(1, 4) ZD_CASE(2, 2) ZD_CASE(2, 3) ZD_CASE(2, 4)
        ZD_CASE(4, 2) ZD_CASE(4, 3) ZD_CASE(4, 4) ZD_CASE(8, 2) ZD_CASE(8, 3) ZD_CASE(8, 4)
#undef ZD_CASE
        if (!fn) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int tz = cfg.tile_z;
        void *args[] = {(void *)&lat, (void *)&g, (void *)&q, (void *)&t, (void *)&seed, (void *)&tz};
        return cudaLaunchKernel(fn, grid, dim3(256), args, smem, s);
    }
    if (cfg.variant == VARIANT_ZFAST) {
        const int W4 = L / 256;
        const dim3 grid((unsigned)((L / (256 / W4)) * (L / cfg.tile_z)), (unsigned)R);
        // programmatic dependent launch (cfg.pdl): the next half-sweep's CTAs are scheduled
        // while this one drains and wait in pdl_enter for its completion
        cudaLaunchConfig_t lc = {};
        lc.gridDim = grid;
        lc.blockDim = dim3(256);
        lc.stream = s;
        cudaLaunchAttribute attr[1] = {pdl_attribute()};
        lc.attrs = attr;
        lc.numAttrs = cfg.pdl ? 1 : 0;
        const int tz = cfg.tile_z;
        switch (W4) {
        case 1: return cudaLaunchKernelEx(&lc, k_sweep_zfast<RULE, 1>, lat, g, q, t, seed, tz);
        case 2: return cudaLaunchKernelEx(&lc, k_sweep_zfast<RULE, 2>, lat, g, q, t, seed, tz);
        case 4: return cudaLaunchKernelEx(&lc, k_sweep_zfast<RULE, 4>, lat, g, q, t, seed, tz);
        default: return cudaLaunchKernelEx(&lc, k_sweep_zfast<RULE, 8>, lat, g, q, t, seed, tz);
        }
    }
    if (cfg.variant == VARIANT_ZMARCH) {
        const int W4 = L / 256;
        const size_t smem = zmarch_smem_bytes(L, cfg.tile_y);
        cudaError_t e =
            cudaFuncSetAttribute(k_sweep_zmarch<RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        const dim3 grid((unsigned)((L / cfg.tile_y) * (L / cfg.tile_z)), (unsigned)R);
        k_sweep_zmarch<RULE><<<grid, cfg.tile_y * W4, smem, s>>>(lat, g, q, t, seed, cfg.tile_y, cfg.tile_z);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)grid_for(g.nw, 256, 8 * (int64_t)device_sms() * 4), (unsigned)R);
    k_sweep_word<RULE><<<grid, 256, 0, s>>>(lat, g, q, t, seed);
    return cudaGetLastError();
}

// Mixed cycle (Supp. Methods I B): sweep t of the lattice keyed S updates blue first when
// bit 0 of word 0 of Philox(counter (0, t, 5, 0), key S) is 1.
int mixed_first(uint64_t S, uint32_t t)
{
    const U4 o = philox4x32_10(0u, t, 5u, 0u, (uint32_t)S, (uint32_t)(S >> 32));
    return (int)(o.x & 1u);
}

template <int RULE>
static cudaError_t sweeps_rule(uint32_t *lat, int L, int R, uint64_t seed, int64_t t0, int64_t n, int cycle,
                               const SweepConfig &cfg, cudaStream_t s, int64_t *launches)
{
    const int64_t nw2 = 2 * make_geom(L).nw;
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        if (cycle == 0) {  // 01 cycle: red, then blue, all replicas in one launch each
            for (int q = 0; q < 2; ++q) {
                cudaError_t e = half_sweep_rule<RULE>(lat, L, R, seed, q, t, cfg, s);
                if (e != cudaSuccess) return e;
            }
            if (launches) *launches += 2;
        } else {           // mixed cycle: each replica its own order
            for (int r = 0; r < R; ++r) {
                const uint64_t S = seed + (uint64_t)r;
                const int first = mixed_first(S, t);
                for (int h = 0; h < 2; ++h) {
                    cudaError_t e = half_sweep_rule<RULE>(lat + (int64_t)r * nw2, L, 1, S, first ^ h, t, cfg, s);
                    if (e != cudaSuccess) return e;
                }
            }
            if (launches) *launches += 2 * R;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_sweeps_packed(uint32_t *lat, int L, int R, uint64_t seed, int rule, int64_t t0, int64_t n,
                                 int cycle, const SweepConfig &cfg, cudaStream_t s, int64_t *launches)
{
    if (n <= 0) return cudaSuccess;
    switch (rule) {
    case TIE_GLAUBER: return sweeps_rule<TIE_GLAUBER>(lat, L, R, seed, t0, n, cycle, cfg, s, launches);
    case TIE_ALWAYS: return sweeps_rule<TIE_ALWAYS>(lat, L, R, seed, t0, n, cycle, cfg, s, launches);
    default: return sweeps_rule<TIE_NEVER>(lat, L, R, seed, t0, n, cycle, cfg, s, launches);
    }
}

// ---------------------------------------------------------------------------------
// Menger-sponge start (Results, the sponge test): the lattice is tiled with sponges of
// iteration k and side 3^k (tiles cut at the lattice edge).  A cell belongs to the sponge
// unless at some base-3 digit position at least two of its coordinates' digits are 1;
// sponge cells take the tile's random sign, the removed cells the opposite one.  Tile
// T = tx + nT*(ty + nT*tz) has sign +1 when bit (T & 31) of word ((T >> 5) & 3) of
// Philox(counter (T >> 7, 0, 4, 0), key S) is set.
__device__ __forceinline__ bool menger_member(int a, int b, int c, int k)
{
    for (int d = 0; d < k; ++d) {
        const int ones = (a % 3 == 1) + (b % 3 == 1) + (c % 3 == 1);
        if (ones >= 2) return false;
        a /= 3;
        b /= 3;
        c /= 3;
    }
    return true;
}

__global__ void k_init_menger(uint32_t *lat, Geom g, uint64_t seed, int k, int side, int nT)
{
    const int r = blockIdx.y, q = blockIdx.z;
    uint32_t *Sq = lat + (2 * (int64_t)r + q) * g.nw;
    const uint64_t S = seed + (uint64_t)r;
    const int L = g.L;
    for (int64_t sw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sw < g.nw;
         sw += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = sw / g.W;
        const int kw = (int)(sw - row * g.W);
        const int y = (int)(row % L), z = (int)(row / L);
        const int p = (y + z + q) & 1;
        uint32_t word = 0u;
        int64_t Tc = -1;
        int sigma = 1;
        for (int b = 0; b < g.RB; ++b) {
            const int x = 2 * (32 * kw + b) + p;
            const int64_t T = x / side + (int64_t)nT * (y / side + (int64_t)nT * (z / side));
            if (T != Tc) {
                const U4 o = philox4x32_10((uint32_t)(T >> 7), 0u, 4u, 0u, (uint32_t)S, (uint32_t)(S >> 32));
                sigma = ((pick(o, (int)((T >> 5) & 3)) >> (T & 31)) & 1u) ? 1 : -1;
                Tc = T;
            }
            const bool in = menger_member(x % side, y % side, z % side, k);
            if ((in ? sigma : -sigma) > 0) word |= 1u << b;
        }
        Sq[sw] = word;
    }
}

cudaError_t launch_init_menger(uint32_t *lat, int L, int R, uint64_t seed, int k, cudaStream_t s)
{
    const Geom g = make_geom(L);
    int side = 1;
    for (int d = 0; d < k; ++d) side *= 3;
    const int nT = (L + side - 1) / side;
    dim3 grid(grid_for(g.nw, 256, 65535), R, 2);
    k_init_menger<<<grid, 256, 0, s>>>(lat, g, seed, k, side, nT);
    return cudaGetLastError();
}

}  // namespace ising
