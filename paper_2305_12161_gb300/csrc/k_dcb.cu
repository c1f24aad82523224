// Double-checkerboard update on the packed store (Supp. Methods I A, after Weigel's GPU
// scheme, in d = 3).  The lattice is cut into blocks; all blocks of one colour run in one
// launch, one CTA per block.  A CTA stages its block and the block's halo (both
// sublattices) in shared memory, updates the block's sites of the first parity there,
// synchronises, and updates the sites of the other parity from the new values.  Blocks of
// one colour never share a face, and the halo belongs to blocks of the other colour, which
// do not change during the launch, so the CTAs are independent.
//
// Per sweep the lattice is read once (plus the halo) and written once: 2 x N/8 bytes plus
// the halo rows, against 3 x N/8 for the two half-sweeps of the plain checkerboard.
//
// Shared-memory layout per sublattice: (by+2) x (bz+2) block rows of rs words (row yy, zz
// holds lattice row (y0-1+yy, z0-1+zz)); the block's own words start at `off`; with an
// x-halo the words at off-1 and off+m are the neighbouring blocks' edge words.  Corner rows
// are never read.  When a block spans an axis (by = L or bz = L) its rows wrap onto
// themselves along that axis and no halo rows are loaded.
#include "common.cuh"
#include "kernels.h"

namespace ising {

namespace {

__device__ __forceinline__ void dcb_cp4(uint32_t *smem, const uint32_t *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void dcb_cp16(uint32_t *smem, const uint32_t *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void dcb_cp_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Parity updated first by block beta in sweep t of the mixed cycle: bit (beta & 31) of word
// ((beta >> 5) & 3) of Philox(counter (beta >> 7, t, 6, 0), key S).
__device__ __forceinline__ int dcb_fine_first(uint64_t S, uint32_t t, int64_t beta)
{
    const U4 o = philox4x32_10((uint32_t)(beta >> 7), t, 6u, 0u, (uint32_t)S, (uint32_t)(S >> 32));
    return (int)((pick(o, (int)((beta >> 5) & 3)) >> (beta & 31)) & 1u);
}

__device__ __forceinline__ int wrap_row(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

}  // namespace

constexpr int DCB_THREADS = 256;
constexpr size_t DCB_SMEM_MAX = 227 * 1024 - 64;

size_t dcb_smem_bytes(const DcbGeom &d)
{
    return 2 * (size_t)(d.by + 2) * (size_t)(d.bz + 2) * (size_t)d.rs * sizeof(uint32_t);
}

static bool axis_ok(int L, int b)
{
    if (b < 1 || b > L || L % b != 0) return false;
    const int nb = L / b;
    return nb == 1 || nb % 2 == 0;
}

bool make_dcb_geom(int L, int bx, int by, int bz, DcbGeom *d)
{
    const Geom g = make_geom(L);
    if (bx == 0) bx = L;
    if (by == 0) by = L <= 16 ? L : 16;
    if (bz == 0) bz = L <= 16 ? L : 8;
    if (!axis_ok(L, by) || !axis_ok(L, bz)) return false;
    if (bx != L && (L < 128 || bx % 64 != 0 || !axis_ok(L, bx))) return false;
    DcbGeom r;
    r.bx = bx;
    r.by = by;
    r.bz = bz;
    r.nbx = L / bx;
    r.nby = L / by;
    r.nbz = L / bz;
    r.xh = bx < L ? 1 : 0;
    r.m = r.xh ? bx / 64 : g.W;
    r.v = (r.m % 4 == 0) ? 4 : 1;
    if (!r.xh) {
        r.off = 0;
        r.rs = r.m;
    } else if (r.v == 4) {  // keep the own words 16-byte aligned
        r.off = 4;
        r.rs = r.m + 8;
    } else {
        r.off = 1;
        r.rs = r.m + 2;
    }
    r.nblk = (int64_t)r.nbx * r.nby * r.nbz;
    if (r.m / r.v + 2 > DCB_THREADS) return false;
    if (dcb_smem_bytes(r) > DCB_SMEM_MAX) return false;
    *d = r;
    return true;
}

// Neighbour word along x that is not at the same compressed index: bit 31 of the previous
// word (p = 0) or bit 0 of the next word (p = 1) of the other sublattice's row.
__device__ __forceinline__ uint4 x_neighbours4(const uint4 &C, uint32_t edge, int p)
{
    uint4 X;
    if (p == 0) {
        X.x = (C.x << 1) | (edge >> 31);
        X.y = (C.y << 1) | (C.x >> 31);
        X.z = (C.z << 1) | (C.y >> 31);
        X.w = (C.w << 1) | (C.z >> 31);
    } else {
        X.x = (C.x >> 1) | (C.y << 31);
        X.y = (C.y >> 1) | (C.z << 31);
        X.z = (C.z >> 1) | (C.w << 31);
        X.w = (C.w >> 1) | (edge << 31);
    }
    return X;
}

// One launch = every block of `colour` (grid.x) for replicas rep0 .. rep0 + grid.y - 1.
// V = words per thread (4: one Philox call per thread covers its words).
template <int RULE, int V>
__global__ void __launch_bounds__(DCB_THREADS) k_sweep_dcb(uint32_t *lat, Geom g, DcbGeom d, int colour,
                                                            uint32_t t, uint64_t seed, int mixed, int rep0)
{
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ int s_f0;
    const int L = g.L, W = g.W;
    const int r = rep0 + (int)blockIdx.y;
    const uint64_t S = seed + (uint64_t)r;
    uint32_t *lat_r = lat + 2 * (int64_t)r * g.nw;

    // The blockIdx.x-th block of this colour: blocks 2i and 2i+1 are neighbours along the
    // first axis that is cut (its block count is even), so exactly one has the colour.
    int64_t beta = d.nblk == 1 ? 0 : 2 * (int64_t)blockIdx.x;
    int bi = (int)(beta % d.nbx), bj = (int)((beta / d.nbx) % d.nby);
    int bk = (int)(beta / ((int64_t)d.nbx * d.nby));
    if (d.nblk > 1 && ((bi + bj + bk) & 1) != colour) {
        ++beta;
        bi = (int)(beta % d.nbx);
        bj = (int)((beta / d.nbx) % d.nby);
        bk = (int)(beta / ((int64_t)d.nbx * d.nby));
    }
    const int m = d.m, rs = d.rs, off = d.off, by = d.by, bz = d.bz;
    const int kw0 = bi * m, y0 = bj * by, z0 = bk * bz;
    const int RY = by + 2, RZ = bz + 2;
    const bool yh = by < L, zh = bz < L;
    const int tid = threadIdx.x;
    if (tid == 0) s_f0 = mixed ? dcb_fine_first(S, t, beta) : 1;
    uint32_t *sm0 = dsm, *sm1 = dsm + RY * RZ * rs;

    // Stage both sublattices' block rows and halo rows: `ch` copy units per row (the own
    // words in V-word units, then the two x-halo words), rows spread over the threads.
    const int own_ch = m / V;
    const int ch = own_ch + 2 * d.xh;
    const int rows_per_iter = DCB_THREADS / ch;
    if (tid < rows_per_iter * ch) {
        const int c = tid % ch;
        for (int rr = tid / ch; rr < 2 * RY * RZ; rr += rows_per_iter) {
            const int a = rr >= RY * RZ ? 1 : 0;
            const int slot = rr - a * RY * RZ;
            const int zz = slot / RY, yy = slot - zz * RY;
            const bool yhal = yy == 0 || yy == RY - 1, zhal = zz == 0 || zz == RZ - 1;
            if ((yhal && (zhal || !yh)) || (zhal && !zh)) continue;  // corners; spanned axes
            if ((yhal || zhal) && c >= own_ch) continue;             // halo rows: own x-range only
            const int y = wrap_row(y0 - 1 + yy, L), z = wrap_row(z0 - 1 + zz, L);
            const uint32_t *grow = lat_r + (int64_t)a * g.nw + ((int64_t)z * L + y) * W;
            uint32_t *srow = (a ? sm1 : sm0) + slot * rs;
            if (c < own_ch) {
                if (V == 4)
                    dcb_cp16(srow + off + 4 * c, grow + kw0 + 4 * c);
                else
                    dcb_cp4(srow + off + c, grow + kw0 + c);
            } else if (c == own_ch) {
                dcb_cp4(srow + off - 1, grow + (kw0 == 0 ? W - 1 : kw0 - 1));
            } else {
                dcb_cp4(srow + off + m, grow + (kw0 + m == W ? 0 : kw0 + m));
            }
        }
    }
    dcb_cp_wait_all();
    __syncthreads();
    const int f0 = s_f0;
    const uint32_t k0 = (uint32_t)S, k1 = (uint32_t)(S >> 32);

    for (int pass = 0; pass < 2; ++pass) {
        const int q = pass == 0 ? f0 : 1 - f0;
        const uint32_t *O = q ? sm0 : sm1;  // the other sublattice: all six neighbours
        uint32_t *Q = q ? sm1 : sm0;
        uint32_t *gQ = lat_r + (int64_t)q * g.nw;
        const int nitems = by * bz * own_ch;
        for (int e = tid; e < nitems; e += DCB_THREADS) {
            const int ro = e / own_ch, cc = e - ro * own_ch;
            const int zo = ro / by, yo = ro - zo * by;
            const int y = y0 + yo, z = z0 + zo;
            const int p = (y + z + q) & 1;
            const int slot = (zo + 1) * RY + (yo + 1);
            const int sym = (!yh && yo == 0) ? slot + (by - 1) : slot - 1;
            const int syp = (!yh && yo == by - 1) ? slot - (by - 1) : slot + 1;
            const int szm = (!zh && zo == 0) ? slot + (bz - 1) * RY : slot - RY;
            const int szp = (!zh && zo == bz - 1) ? slot - (bz - 1) * RY : slot + RY;
            const int64_t sw0 = ((int64_t)z * L + y) * W + kw0 + V * cc;
            if (V == 4) {
                const int w = off + 4 * cc;
                const uint4 C = *reinterpret_cast<const uint4 *>(O + slot * rs + w);
                const uint4 Ym = *reinterpret_cast<const uint4 *>(O + sym * rs + w);
                const uint4 Yp = *reinterpret_cast<const uint4 *>(O + syp * rs + w);
                const uint4 Zm = *reinterpret_cast<const uint4 *>(O + szm * rs + w);
                const uint4 Zp = *reinterpret_cast<const uint4 *>(O + szp * rs + w);
                const uint4 Sq = *reinterpret_cast<const uint4 *>(Q + slot * rs + w);
                int ei;
                if (p == 0)
                    ei = (cc == 0 && !d.xh) ? m - 1 : 4 * cc - 1;
                else
                    ei = (cc == own_ch - 1 && !d.xh) ? 0 : 4 * cc + 4;
                const uint4 X = x_neighbours4(C, O[slot * rs + off + ei], p);
                uint32_t ge[4], eq[4];
                count6(C.x, X.x, Ym.x, Yp.x, Zm.x, Zp.x, ge[0], eq[0]);
                count6(C.y, X.y, Ym.y, Yp.y, Zm.y, Zp.y, ge[1], eq[1]);
                count6(C.z, X.z, Ym.z, Yp.z, Zm.z, Zp.z, ge[2], eq[2]);
                count6(C.w, X.w, Ym.w, Yp.w, Zm.w, Zp.w, ge[3], eq[3]);
                U4 rnd{0u, 0u, 0u, 0u};
                if (RULE == TIE_GLAUBER && (eq[0] | eq[1] | eq[2] | eq[3]) != 0u)
                    rnd = philox4x32_10((uint32_t)(sw0 >> 2), t, (uint32_t)q, 0u, k0, k1);
                uint4 nw;
                nw.x = resolve<RULE>(Sq.x, ge[0], eq[0], rnd.x);
                nw.y = resolve<RULE>(Sq.y, ge[1], eq[1], rnd.y);
                nw.z = resolve<RULE>(Sq.z, ge[2], eq[2], rnd.z);
                nw.w = resolve<RULE>(Sq.w, ge[3], eq[3], rnd.w);
                if (pass == 0) *reinterpret_cast<uint4 *>(Q + slot * rs + w) = nw;
                *reinterpret_cast<uint4 *>(gQ + sw0) = nw;
            } else {
                const int w = off + cc;
                const uint32_t C = O[slot * rs + w];
                uint32_t X;
                if (m == 1 && !d.xh) {  // the whole row is one word (L <= 64): wrap inside it
                    const int RB = g.RB;
                    X = p == 0 ? (((C << 1) | (C >> (RB - 1))) & row_mask(RB)) : ((C >> 1) | ((C & 1u) << (RB - 1)));
                } else if (p == 0) {
                    const int ei = (cc == 0 && !d.xh) ? m - 1 : cc - 1;
                    X = (C << 1) | (O[slot * rs + off + ei] >> 31);
                } else {
                    const int ei = (cc == m - 1 && !d.xh) ? 0 : cc + 1;
                    X = (C >> 1) | (O[slot * rs + off + ei] << 31);
                }
                uint32_t ge4, eq3;
                count6(C, X, O[sym * rs + w], O[syp * rs + w], O[szm * rs + w], O[szp * rs + w], ge4, eq3);
                uint32_t rnd = 0u;
                if (RULE == TIE_GLAUBER && eq3 != 0u) rnd = rng_word(g, sw0, t, (uint32_t)q, S);
                const uint32_t nw = resolve<RULE>(Q[slot * rs + w], ge4, eq3, rnd);
                if (pass == 0) Q[slot * rs + w] = nw;
                gQ[sw0] = nw;
            }
        }
        if (pass == 0) __syncthreads();
    }
}

// Full-row blocks of a lattice whose rows are W4 = L/256 uint4 units (L = 256 .. 2048):
// the same algorithm with the row width a compile-time constant, the thread's unit and
// first row fixed for the whole kernel and rows advanced by increments (no divisions),
// and the Philox round keys computed once per thread.
template <int RULE, int W4>
__global__ void __launch_bounds__(DCB_THREADS) k_sweep_dcb_rows(uint32_t *lat, Geom g, DcbGeom d, int colour,
                                                                 uint32_t t, uint64_t seed, int mixed, int rep0)
{
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ int s_f0;
    constexpr int M = 4 * W4;                // words per row and sublattice
    constexpr int RPI = DCB_THREADS / W4;    // rows handled per pass over the threads
    const int L = g.L;
    const int r = rep0 + (int)blockIdx.y;
    const uint64_t S = seed + (uint64_t)r;
    uint32_t *lat_r = lat + 2 * (int64_t)r * g.nw;

    int64_t beta = d.nblk == 1 ? 0 : 2 * (int64_t)blockIdx.x;
    int bj = (int)(beta % d.nby), bk = (int)(beta / d.nby);  // nbx = 1
    if (d.nblk > 1 && ((bj + bk) & 1) != colour) {
        ++beta;
        bj = (int)(beta % d.nby);
        bk = (int)(beta / d.nby);
    }
    const int by = d.by, bz = d.bz;
    const int y0 = bj * by, z0 = bk * bz;
    const int RY = by + 2, RZ = bz + 2;
    const bool yh = by < L, zh = bz < L;
    const int tid = threadIdx.x;
    const int c = tid % W4;    // this thread's uint4 unit of every row it touches
    const int r0 = tid / W4;   // its first row
    if (tid == 0) s_f0 = mixed ? dcb_fine_first(S, t, beta) : 1;
    uint4 *const smA = reinterpret_cast<uint4 *>(dsm);
    uint4 *const smB = smA + RY * RZ * W4;
    const uint4 *const gA = reinterpret_cast<const uint4 *>(lat_r);
    const uint4 *const gB = reinterpret_cast<const uint4 *>(lat_r + g.nw);

    // Stage: slots of the (RY x RZ) row grid, corner rows and spanned-axis halos skipped.
    {
        int yy = r0 % RY, zz = r0 / RY;
        for (int slot = r0; slot < RY * RZ; slot += RPI) {
            const bool yhal = yy == 0 || yy == RY - 1, zhal = zz == 0 || zz == RZ - 1;
            if (!((yhal && (zhal || !yh)) || (zhal && !zh))) {
                const int y = wrap_row(y0 - 1 + yy, L), z = wrap_row(z0 - 1 + zz, L);
                const int64_t gi = ((int64_t)z * L + y) * W4 + c;
                dcb_cp16(reinterpret_cast<uint32_t *>(smA + slot * W4 + c), reinterpret_cast<const uint32_t *>(gA + gi));
                dcb_cp16(reinterpret_cast<uint32_t *>(smB + slot * W4 + c), reinterpret_cast<const uint32_t *>(gB + gi));
            }
            yy += RPI;
            while (yy >= RY) {
                yy -= RY;
                ++zz;
            }
        }
    }
    const PhiloxKeys keys = philox_keys(S);
    dcb_cp_wait_all();
    __syncthreads();
    const int f0 = s_f0;

    for (int pass = 0; pass < 2; ++pass) {
        const int q = pass == 0 ? f0 : 1 - f0;
        const uint4 *O = q ? smA : smB;
        uint4 *Q = q ? smB : smA;
        uint4 *gQ = reinterpret_cast<uint4 *>(lat_r + (int64_t)q * g.nw);
        int yo = r0 % by, zo = r0 / by;
        for (int ro = r0; ro < by * bz; ro += RPI) {
            const int y = y0 + yo, z = z0 + zo;
            const int p = (y + z + q) & 1;
            const int slot = (zo + 1) * RY + (yo + 1);
            const int sym = (!yh && yo == 0) ? slot + (by - 1) : slot - 1;
            const int syp = (!yh && yo == by - 1) ? slot - (by - 1) : slot + 1;
            const int szm = (!zh && zo == 0) ? slot + (bz - 1) * RY : slot - RY;
            const int szp = (!zh && zo == bz - 1) ? slot - (bz - 1) * RY : slot + RY;
            const uint4 C = O[slot * W4 + c];
            const uint4 Ym = O[sym * W4 + c];
            const uint4 Yp = O[syp * W4 + c];
            const uint4 Zm = O[szm * W4 + c];
            const uint4 Zp = O[szp * W4 + c];
            const uint4 Sq = Q[slot * W4 + c];
            const uint32_t *Orow = reinterpret_cast<const uint32_t *>(O + slot * W4);
            const int ei = p == 0 ? (c == 0 ? M - 1 : 4 * c - 1) : (c == W4 - 1 ? 0 : 4 * c + 4);
            const uint4 X = x_neighbours4(C, Orow[ei], p);
            uint32_t ge[4], eq[4];
            count6(C.x, X.x, Ym.x, Yp.x, Zm.x, Zp.x, ge[0], eq[0]);
            count6(C.y, X.y, Ym.y, Yp.y, Zm.y, Zp.y, ge[1], eq[1]);
            count6(C.z, X.z, Ym.z, Yp.z, Zm.z, Zp.z, ge[2], eq[2]);
            count6(C.w, X.w, Ym.w, Yp.w, Zm.w, Zp.w, ge[3], eq[3]);
            const int64_t u = ((int64_t)z * L + y) * W4 + c;  // uint4 index = Philox counter word
            U4 rnd{0u, 0u, 0u, 0u};
            if (RULE == TIE_GLAUBER && (eq[0] | eq[1] | eq[2] | eq[3]) != 0u)
                rnd = philox4x32_10_rk((uint32_t)u, t, (uint32_t)q, 0u, keys);
            uint4 nw;
            nw.x = resolve<RULE>(Sq.x, ge[0], eq[0], rnd.x);
            nw.y = resolve<RULE>(Sq.y, ge[1], eq[1], rnd.y);
            nw.z = resolve<RULE>(Sq.z, ge[2], eq[2], rnd.z);
            nw.w = resolve<RULE>(Sq.w, ge[3], eq[3], rnd.w);
            if (pass == 0) Q[slot * W4 + c] = nw;
            gQ[u] = nw;
            yo += RPI;
            while (yo >= by) {
                yo -= by;
                ++zo;
            }
        }
        if (pass == 0) __syncthreads();
    }
}

template <int RULE, int W4>
static cudaError_t dcb_rows_rule(uint32_t *lat, const Geom &g, int R, uint64_t seed, int64_t t0, int64_t n,
                                 int cycle, const DcbGeom &d, cudaStream_t s, int64_t *launches)
{
    const size_t smem = dcb_smem_bytes(d);
    cudaError_t e =
        cudaFuncSetAttribute(k_sweep_dcb_rows<RULE, W4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t per_colour[2] = {d.nblk == 1 ? 1 : d.nblk / 2, d.nblk == 1 ? 0 : d.nblk / 2};
    int64_t nl = 0;
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        if (cycle == 0) {
            for (int colour = 0; colour < 2; ++colour) {
                if (per_colour[colour] == 0) continue;
                k_sweep_dcb_rows<RULE, W4><<<dim3((unsigned)per_colour[colour], (unsigned)R), DCB_THREADS, smem, s>>>(
                    lat, g, d, colour, t, seed, 0, 0);
                ++nl;
            }
        } else {
            for (int r = 0; r < R; ++r) {
                const int first = mixed_first(seed + (uint64_t)r, t);
                for (int pass = 0; pass < 2; ++pass) {
                    const int colour = first ^ pass;
                    if (per_colour[colour] == 0) continue;
                    k_sweep_dcb_rows<RULE, W4><<<dim3((unsigned)per_colour[colour], 1u), DCB_THREADS, smem, s>>>(
                        lat, g, d, colour, t, seed, 1, r);
                    ++nl;
                }
            }
        }
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

template <int RULE, int V>
static cudaError_t dcb_rule(uint32_t *lat, const Geom &g, int R, uint64_t seed, int64_t t0, int64_t n, int cycle,
                            const DcbGeom &d, cudaStream_t s, int64_t *launches)
{
    const size_t smem = dcb_smem_bytes(d);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_dcb<RULE, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // Blocks per colour: half of them, or the single block (red) when no axis is cut.
    const int64_t per_colour[2] = {d.nblk == 1 ? 1 : d.nblk / 2, d.nblk == 1 ? 0 : d.nblk / 2};
    int64_t nl = 0;
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        if (cycle == 0) {
            for (int colour = 0; colour < 2; ++colour) {
                if (per_colour[colour] == 0) continue;
                k_sweep_dcb<RULE, V><<<dim3((unsigned)per_colour[colour], (unsigned)R), DCB_THREADS, smem, s>>>(
                    lat, g, d, colour, t, seed, 0, 0);
                ++nl;
            }
        } else {  // mixed cycle: each replica its own colour order
            for (int r = 0; r < R; ++r) {
                const int first = mixed_first(seed + (uint64_t)r, t);
                for (int pass = 0; pass < 2; ++pass) {
                    const int colour = first ^ pass;
                    if (per_colour[colour] == 0) continue;
                    k_sweep_dcb<RULE, V><<<dim3((unsigned)per_colour[colour], 1u), DCB_THREADS, smem, s>>>(
                        lat, g, d, colour, t, seed, 1, r);
                    ++nl;
                }
            }
        }
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

template <int RULE>
static cudaError_t dcb_rule_v(uint32_t *lat, const Geom &g, int R, uint64_t seed, int64_t t0, int64_t n, int cycle,
                              const DcbGeom &d, cudaStream_t s, int64_t *launches)
{
    if (!d.xh) {
        switch (g.L) {
        case 256: return dcb_rows_rule<RULE, 1>(lat, g, R, seed, t0, n, cycle, d, s, launches);
        case 512: return dcb_rows_rule<RULE, 2>(lat, g, R, seed, t0, n, cycle, d, s, launches);
        case 1024: return dcb_rows_rule<RULE, 4>(lat, g, R, seed, t0, n, cycle, d, s, launches);
        case 2048: return dcb_rows_rule<RULE, 8>(lat, g, R, seed, t0, n, cycle, d, s, launches);
        default: break;
        }
    }
    if (d.v == 4) return dcb_rule<RULE, 4>(lat, g, R, seed, t0, n, cycle, d, s, launches);
    return dcb_rule<RULE, 1>(lat, g, R, seed, t0, n, cycle, d, s, launches);
}

cudaError_t launch_sweeps_dcb(uint32_t *lat, int L, int R, uint64_t seed, int rule, int64_t t0, int64_t n_mcs,
                              int cycle, const DcbGeom &d, cudaStream_t s, int64_t *launches)
{
    if (n_mcs <= 0) return cudaSuccess;
    const Geom g = make_geom(L);
    switch (rule) {
    case TIE_GLAUBER: return dcb_rule_v<TIE_GLAUBER>(lat, g, R, seed, t0, n_mcs, cycle, d, s, launches);
    case TIE_ALWAYS: return dcb_rule_v<TIE_ALWAYS>(lat, g, R, seed, t0, n_mcs, cycle, d, s, launches);
    default: return dcb_rule_v<TIE_NEVER>(lat, g, R, seed, t0, n_mcs, cycle, d, s, launches);
    }
}

}  // namespace ising
