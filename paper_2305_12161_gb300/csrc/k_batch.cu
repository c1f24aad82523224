// Batched form: many independent lattices of uneven L advanced by ONE persistent
// cooperative launch per run segment (n MCS between two measurements).
//
// Work list, one entry per CTA (built on the host, balanced by expected cost):
//   LOCAL  — the CTA owns whole small lattices (packed state <= its shared memory, e.g.
//            64^3 = 32 KiB).  It loads one into shared memory, runs all n MCS there with
//            __syncthreads between half-sweeps, writes it back, and takes the next.
//            No HBM traffic inside the segment.
//   GROUP  — the CTA is rank k of a group of CTAs that share one larger lattice, each
//            updating a contiguous slab of its Philox groups (z-major, so a slab is a
//            run of planes).  Between half-sweeps the group meets at a barrier in
//            global memory; its spin is bounded by %globaltimer and a timeout sets the
//            batch's status word instead of hanging.  Loads bypass L1 (ld.global.cg), as
//            other CTAs write the lattice inside the launch; the batch's larger lattices
//            together fit in L2.
// The update rule, the neighbour words and the random bits are those of the single-
// lattice kernels (common.cuh), so every lattice follows exactly its single-run
// trajectory.
#include "common.cuh"
#include "kernels.h"
#include "batch.h"

namespace ising {

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Loads of neighbour words: from shared memory (plain) or from global memory through
// L2 only (the lattice is written by other CTAs during the launch).
struct FromShared {
    __device__ __forceinline__ static uint32_t ld(const uint32_t *p) { return *p; }
    __device__ __forceinline__ static uint4 ld4(const uint4 *p) { return *p; }
    __device__ __forceinline__ static uint2 ld2(const uint2 *p) { return *p; }
};
struct FromL2 {
    __device__ __forceinline__ static uint32_t ld(const uint32_t *p) { return __ldcg(p); }
    __device__ __forceinline__ static uint4 ld4(const uint4 *p) { return __ldcg(p); }
    __device__ __forceinline__ static uint2 ld2(const uint2 *p) { return __ldcg(p); }
};

template <class LD>
__device__ __forceinline__ Nbrs nbrs_of(const uint32_t *O, const Geom &g, int64_t sw, int q)
{
    const int L = g.L, W = g.W;
    const int64_t row = sw / W;
    const int kw = (int)(sw - row * W);
    const int y = (int)(row % L);
    const int z = (int)(row / L);
    const int p = (y + z + q) & 1;
    Nbrs n;
    n.C = LD::ld(O + sw);
    if (W >= 2) {
        if (p == 0)
            n.X = (n.C << 1) | (LD::ld(O + row * W + (kw == 0 ? W - 1 : kw - 1)) >> 31);
        else
            n.X = (n.C >> 1) | (LD::ld(O + row * W + (kw == W - 1 ? 0 : kw + 1)) << 31);
    } else {
        const int RB = g.RB;
        if (p == 0)
            n.X = ((n.C << 1) | (n.C >> (RB - 1))) & row_mask(RB);
        else
            n.X = (n.C >> 1) | ((n.C & 1u) << (RB - 1));
    }
    const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
    n.Ym = LD::ld(O + ((int64_t)z * L + ym) * W + kw);
    n.Yp = LD::ld(O + ((int64_t)z * L + yp) * W + kw);
    n.Zm = LD::ld(O + ((int64_t)zm * L + y) * W + kw);
    n.Zp = LD::ld(O + ((int64_t)zp * L + y) * W + kw);
    return n;
}

// Resolve four words of one Philox group and return them.
template <int RULE>
__device__ __forceinline__ uint4 resolve4(const uint4 &s, const uint32_t ge[4], const uint32_t eq[4], uint32_t unit,
                                          uint32_t t, int q, uint64_t key)
{
    U4 o{0u, 0u, 0u, 0u};
    if (RULE == TIE_GLAUBER && (eq[0] | eq[1] | eq[2] | eq[3]))
        o = philox4x32_10((uint32_t)unit, t, (uint32_t)q, 0u, (uint32_t)key, (uint32_t)(key >> 32));
    return make_uint4(resolve<RULE>(s.x, ge[0], eq[0], o.x), resolve<RULE>(s.y, ge[1], eq[1], o.y),
                      resolve<RULE>(s.z, ge[2], eq[2], o.z), resolve<RULE>(s.w, ge[3], eq[3], o.w));
}

__device__ __forceinline__ uint32_t xshift(uint32_t c, uint32_t edge_prev, uint32_t edge_next, int p)
{
    return p == 0 ? __funnelshift_l(edge_prev, c, 1) : __funnelshift_r(c, edge_next, 1);
}

// Update one unit (the 4 words of one Philox group) of sublattice q in place.
//   W >= 4 (L >= 256): the unit is one uint4 inside a row; neighbour rows are uint4 loads.
//   W == 2 (L = 128):  the unit is two whole rows of two words.
//   W == 1 (L = 64):   the unit is four whole one-word rows y..y+3 of one plane; the
//                      y-neighbours are the same vector shifted by one row plus the
//                      edge words of rows y-1 and y+4.
//   L < 64:            one padded row word per unit (rows of L/2 sites).
template <int RULE, class LD>
__device__ __forceinline__ void update_unit(uint32_t *Sq, const uint32_t *O, const Geom &g, int64_t unit, int q,
                                            uint32_t t, uint64_t key)
{
    const int L = g.L, W = g.W;
    const uint4 *O4 = reinterpret_cast<const uint4 *>(O);
    uint4 *S4 = reinterpret_cast<uint4 *>(Sq);
    uint32_t ge[4], eq[4];
    if (L % 256 == 0) {
        const int W4 = W >> 2;
        const int64_t row = unit / W4;
        const int c4 = (int)(unit - row * W4);
        const int y = (int)(row % L), z = (int)(row / L);
        const int p = (y + z + q) & 1;
        const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
        const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
        const uint4 c = LD::ld4(O4 + unit);
        const uint4 a = LD::ld4(O4 + ((int64_t)z * L + ym) * W4 + c4);
        const uint4 b = LD::ld4(O4 + ((int64_t)z * L + yp) * W4 + c4);
        const uint4 d = LD::ld4(O4 + ((int64_t)zm * L + y) * W4 + c4);
        const uint4 e = LD::ld4(O4 + ((int64_t)zp * L + y) * W4 + c4);
        uint32_t edge;
        if (p == 0) edge = LD::ld(O + row * W + ((c4 == 0 ? W4 : c4) * 4 - 1));
        else edge = LD::ld(O + row * W + (c4 == W4 - 1 ? 0 : c4 * 4 + 4));
        count6(c.x, xshift(c.x, edge, c.y, p), a.x, b.x, d.x, e.x, ge[0], eq[0]);
        count6(c.y, xshift(c.y, c.x, c.z, p), a.y, b.y, d.y, e.y, ge[1], eq[1]);
        count6(c.z, xshift(c.z, c.y, c.w, p), a.z, b.z, d.z, e.z, ge[2], eq[2]);
        count6(c.w, xshift(c.w, c.z, edge, p), a.w, b.w, d.w, e.w, ge[3], eq[3]);
        S4[unit] = resolve4<RULE>(LD::ld4(S4 + unit), ge, eq, (uint32_t)unit, t, q, key);
    } else if (L == 128) {
        // rows r, r+1 (y, y+1 of one plane: L is even), words (kw 0, kw 1) each
        const int64_t row = unit * 2;
        const int y = (int)(row % L), z = (int)(row / L);
        const uint2 *O2 = reinterpret_cast<const uint2 *>(O);
        const uint4 c = LD::ld4(O4 + unit);
        const int ym = y == 0 ? L - 1 : y - 1, yp2 = y + 2 == L ? 0 : y + 2;
        const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
        const uint2 a = LD::ld2(O2 + (int64_t)z * L + ym);    // row y-1
        const uint2 b = LD::ld2(O2 + (int64_t)z * L + yp2);   // row y+2
        const uint4 d = LD::ld4(O4 + (((int64_t)zm * L + y) >> 1));
        const uint4 e = LD::ld4(O4 + (((int64_t)zp * L + y) >> 1));
        const int p0 = (y + z + q) & 1, p1 = p0 ^ 1;
        // words: x = (row y, kw0), y = (row y, kw1), z = (row y+1, kw0), w = (row y+1, kw1)
        count6(c.x, xshift(c.x, c.y, c.y, p0), a.x, c.z, d.x, e.x, ge[0], eq[0]);
        count6(c.y, xshift(c.y, c.x, c.x, p0), a.y, c.w, d.y, e.y, ge[1], eq[1]);
        count6(c.z, xshift(c.z, c.w, c.w, p1), c.x, b.x, d.z, e.z, ge[2], eq[2]);
        count6(c.w, xshift(c.w, c.z, c.z, p1), c.y, b.y, d.w, e.w, ge[3], eq[3]);
        S4[unit] = resolve4<RULE>(LD::ld4(S4 + unit), ge, eq, (uint32_t)unit, t, q, key);
    } else if (L == 64) {
        // rows y..y+3 of plane z, one word each (a full row is one 32-bit word)
        const int64_t row = unit * 4;
        const int y = (int)(row & 63), z = (int)(row >> 6);
        const int zm = z == 0 ? 63 : z - 1, zp = z == 63 ? 0 : z + 1;
        const uint4 c = LD::ld4(O4 + unit);
        const uint32_t prev = LD::ld(O + (int64_t)z * 64 + (y == 0 ? 63 : y - 1));
        const uint32_t next = LD::ld(O + (int64_t)z * 64 + (y + 4 == 64 ? 0 : y + 4));
        const uint4 d = LD::ld4(O4 + (((int64_t)zm * 64 + y) >> 2));
        const uint4 e = LD::ld4(O4 + (((int64_t)zp * 64 + y) >> 2));
        const int p0 = (y + z + q) & 1, p1 = p0 ^ 1;
        // a row is its own ring: the x edge comes from the same word (rotation)
        count6(c.x, xshift(c.x, c.x, c.x, p0), prev, c.y, d.x, e.x, ge[0], eq[0]);
        count6(c.y, xshift(c.y, c.y, c.y, p1), c.x, c.z, d.y, e.y, ge[1], eq[1]);
        count6(c.z, xshift(c.z, c.z, c.z, p0), c.y, c.w, d.z, e.z, ge[2], eq[2]);
        count6(c.w, xshift(c.w, c.w, c.w, p1), c.z, next, d.w, e.w, ge[3], eq[3]);
        S4[unit] = resolve4<RULE>(LD::ld4(S4 + unit), ge, eq, (uint32_t)unit, t, q, key);
    } else if (L >= 64) {
        // other multiples of 64 (rows of W words, W not a multiple of 4): word by word
        const int64_t sw0 = unit * 4;
        uint4 s;
        uint32_t *sp = reinterpret_cast<uint32_t *>(&s);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const Nbrs n = nbrs_of<LD>(O, g, sw0 + i, q);
            count6(n.C, n.X, n.Ym, n.Yp, n.Zm, n.Zp, ge[i], eq[i]);
            sp[i] = LD::ld(Sq + sw0 + i);
        }
        const uint4 nw = resolve4<RULE>(s, ge, eq, (uint32_t)unit, t, q, key);
        Sq[sw0 + 0] = nw.x;
        Sq[sw0 + 1] = nw.y;
        Sq[sw0 + 2] = nw.z;
        Sq[sw0 + 3] = nw.w;
    } else {
        const Nbrs n = nbrs_of<LD>(O, g, unit, q);
        uint32_t ge1, eq1;
        count6(n.C, n.X, n.Ym, n.Yp, n.Zm, n.Zp, ge1, eq1);
        const uint32_t s = LD::ld(Sq + unit);
        uint32_t rnd = 0u;
        if (RULE == TIE_GLAUBER && eq1) rnd = rng_word(g, unit, t, (uint32_t)q, key);
        Sq[unit] = resolve<RULE>(s, ge1, eq1, rnd);
    }
}

__device__ __forceinline__ int64_t units_of(const Geom &g) { return g.L >= 64 ? g.nw / 4 : g.nw; }

// Group barrier: CTA-wide, generation-counted, bounded wait.  Returns false once the
// batch status is set (by this or another CTA), so every CTA drains quickly.
__device__ bool group_barrier(unsigned *ctr, unsigned members, unsigned gen, int *status, uint64_t timeout_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(ctr, 1u);
        const unsigned target = (gen + 1u) * members;
        const uint64_t t0 = globaltimer_ns();
        while (ld_acquire(ctr) < target) {
            if (*(volatile int *)status != 0) {
                ok = 0;
                break;
            }
            if (globaltimer_ns() - t0 > timeout_ns) {
                atomicCAS(status, 0, BATCH_STATUS_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <int RULE>
__global__ void __launch_bounds__(BATCH_THREADS, 4) k_batch(const BatchTask *__restrict__ tasks,
                                                         const BatchLattice *__restrict__ lats, uint32_t t0, int n_mcs,
                                                         unsigned *barriers, int *status, uint64_t timeout_ns,
                                                         int missing_cta, unsigned long long *cta_ns)
{
    extern __shared__ uint4 bsm4[];
    uint32_t *bsm = reinterpret_cast<uint32_t *>(bsm4);
    const BatchTask task = tasks[blockIdx.x];
    const int tid = threadIdx.x;
    const uint64_t start = globaltimer_ns();
    if ((int)blockIdx.x == missing_cta) return;  // failure injection: this CTA never arrives

    if (task.mode == BATCH_LOCAL) {
        for (int li = task.first; li < task.first + task.count; ++li) {
            const BatchLattice b = lats[li];
            const Geom g = make_geom(b.L);
            const int64_t nw = g.nw;
            uint4 *src4 = reinterpret_cast<uint4 *>(b.lat);
            for (int64_t i = tid; i < (2 * nw) / 4; i += BATCH_THREADS) bsm4[i] = __ldcg(src4 + i);
            __syncthreads();
            const int64_t nu = units_of(g);
            for (int k = 0; k < n_mcs; ++k) {
                const uint32_t t = t0 + (uint32_t)k;
                for (int q = 0; q < 2; ++q) {
                    uint32_t *Sq = bsm + (int64_t)q * nw;
                    const uint32_t *O = bsm + (int64_t)(1 - q) * nw;
                    for (int64_t u = tid; u < nu; u += BATCH_THREADS) {
                        if (RULE == TIE_GLAUBER) update_unit<TIE_GLAUBER, FromShared>(Sq, O, g, u, q, t, b.S);
                        else if (RULE == TIE_ALWAYS) update_unit<TIE_ALWAYS, FromShared>(Sq, O, g, u, q, t, b.S);
                        else update_unit<TIE_NEVER, FromShared>(Sq, O, g, u, q, t, b.S);
                    }
                    __syncthreads();
                }
            }
            for (int64_t i = tid; i < (2 * nw) / 4; i += BATCH_THREADS) src4[i] = bsm4[i];
            __syncthreads();
        }
    } else {
        const BatchLattice b = lats[task.first];
        const Geom g = make_geom(b.L);
        const int64_t nu = units_of(g);
        const int64_t u0 = nu * task.rank / task.size, u1 = nu * (task.rank + 1) / task.size;
        unsigned gen = 0;
        for (int k = 0; k < n_mcs; ++k) {
            const uint32_t t = t0 + (uint32_t)k;
            for (int q = 0; q < 2; ++q) {
                uint32_t *Sq = b.lat + (int64_t)q * g.nw;
                const uint32_t *O = b.lat + (int64_t)(1 - q) * g.nw;
                for (int64_t u = u0 + tid; u < u1; u += BATCH_THREADS) {
                    if (RULE == TIE_GLAUBER) update_unit<TIE_GLAUBER, FromL2>(Sq, O, g, u, q, t, b.S);
                    else if (RULE == TIE_ALWAYS) update_unit<TIE_ALWAYS, FromL2>(Sq, O, g, u, q, t, b.S);
                    else update_unit<TIE_NEVER, FromL2>(Sq, O, g, u, q, t, b.S);
                }
                if (task.size > 1) {
                    if (!group_barrier(barriers + task.group, (unsigned)task.size, gen, status, timeout_ns)) goto done;
                    ++gen;
                } else {
                    __syncthreads();
                }
            }
        }
    }
done:
    if (cta_ns && tid == 0) cta_ns[blockIdx.x] = globaltimer_ns() - start;
}

cudaError_t batch_occupancy(int smem_bytes, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_batch<TIE_GLAUBER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_batch<TIE_ALWAYS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_batch<TIE_NEVER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<TIE_GLAUBER>, BATCH_THREADS, smem_bytes);
    *blocks_per_sm = occ;
    return e;
}

cudaError_t launch_batch(const BatchTask *tasks, int ntasks, const BatchLattice *lats, int rule, uint32_t t0, int n_mcs,
                         unsigned *barriers, int *status, uint64_t timeout_ns, int missing_cta,
                         unsigned long long *cta_ns, int smem_bytes, cudaStream_t s)
{
    void *fn;
    if (rule == TIE_GLAUBER) fn = (void *)k_batch<TIE_GLAUBER>;
    else if (rule == TIE_ALWAYS) fn = (void *)k_batch<TIE_ALWAYS>;
    else fn = (void *)k_batch<TIE_NEVER>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ntasks);
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident: group barriers cannot deadlock
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&tasks, (void *)&lats, (void *)&t0, (void *)&n_mcs, (void *)&barriers,
                    (void *)&status, (void *)&timeout_ns, (void *)&missing_cta, (void *)&cta_ns};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ising
