// Axis correlation sums D_a(r) on the tensor cores.
//
// Along one axis the lattice is L^2 lines of L sites.  With s = +-1,
//   sum_i [s_i != s_(i + r e_a)] = (L * L^2 - S(r)) / 2,   S(r) = sum_j G[j][(j + r) mod L],
// where G[j][k] = sum over lines of s(j) s(k) is the Gram matrix of the L positions over
// the lines: a dense contraction of length L^2.  A packed word holds the same position of
// 32 lines, so one word is the K = 32 slice of one fp8 tcgen05.mma: its bits become e4m3
// values +1 / -1 (exact), products accumulate in fp32, and every partial sum is an even
// integer of magnitude <= L^2 <= 2^24, so the result is exact.
//
// Only the upper block triangle of G is computed (G is symmetric); an entry of an
// off-diagonal tile stands for both ordered pairs (j, k) and (k, j).  Per replica and axis:
// the axis's lines are expanded once into e4m3 rows in one of two scratch halves (x by
// k_expand_x_e4m3; y and z by the helper warps of the previous axis's product, into the
// other half), and k_gram_tma accumulates the 128 x 128 tiles of G by tcgen05.mma in tensor
// memory from TMA-loaded, 128-byte swizzled shared-memory operands; each entry's -G/2 is
// added to D at its cyclic distance; the records start from N/2.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ising {

constexpr int TM_T = 128;        // positions per tile side (M = N = 128)
constexpr int GT_N = 256;        // B rows per CTA: two adjacent 128-position tiles (MMA N = 256)
constexpr int GT_STAGES = 4;     // TMA pipeline depth (48 KB per stage)
constexpr int GT_KB = 128;       // K bytes (= lines) per stage and operand box
constexpr int GT_STAGE_BYTES = (TM_T + GT_N) * GT_KB;
constexpr int UMMA_WAIT_LIMIT = 1 << 30;  // backstop on try_wait rounds (the wall-time bound comes first)
constexpr int GT_THREADS = 256;  // Gram CTA: warps 0-3 load, multiply and read back; 4-7 expand the next axis


// Four e4m3 values from the four bits of n (n < 16): bit i -> byte i, +1.0 (0x38) when
// set, -1.0 (0xB8) when clear.  The multiplier places bit i at bit 8i + 7 (and the other
// bits of n at positions that the mask drops, without carries).
__device__ __forceinline__ uint32_t e4m3x4(uint32_t n)
{
    return ((n * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05.mma for a K-major operand in 128-byte swizzled
// atoms (8 rows x 128 bytes; the 16-byte chunk c of row r stored at chunk c ^ r): start
// address, leading byte offset 16 (unused when K fits one atom row), stride 1024 bytes between
// atoms along M/N, descriptor version 1, swizzle mode 128B.  The K slice of 32 fp8 values at
// byte offset 32 s of the atom row is addressed by starting 32 s bytes later.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: D in f32, A and B e4m3, both K-major, M = 128, N = GT_N.
constexpr uint32_t UMMA_IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(GT_N >> 3) << 17) |
                                ((uint32_t)(TM_T >> 4) << 24);

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier for at most timeout_ns of wall time (and at most
// UMMA_WAIT_LIMIT rounds); false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, uint64_t timeout_ns)
{
    const uint64_t t0 = globaltimer_ns();
    for (int it = 0; it < UMMA_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255) == 255 && globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// ---------------------------------------------------------------------------------
// The Gram products run on operands expanded once per measurement: E holds, for every
// position p of the axis and every line K of it, the e4m3 value of s (+1 -> 0x38, -1 -> 0xB8),
// chunk-major: the 128 lines of chunk K/128 of all L positions are one block of L x 128 bytes,
// E[(K / 128) * L * 128 + p * 128 + K % 128], so a box of 128 positions x 128 lines is 16
// contiguous KB (rows L^2 bytes apart would put every box's rows at a large power-of-two
// stride).  Column cc of the panels (32 lines) is K = 32 cc .. 32 cc + 31.  Every word of the
// lattice is expanded once instead of once per tile pair.
__device__ __forceinline__ void expand_e4m3_word(uint32_t v, uint4 &lo, uint4 &hi)
{
    lo.x = e4m3x4(v & 0xFu);
    lo.y = e4m3x4((v >> 4) & 0xFu);
    lo.z = e4m3x4((v >> 8) & 0xFu);
    lo.w = e4m3x4((v >> 12) & 0xFu);
    hi.x = e4m3x4((v >> 16) & 0xFu);
    hi.y = e4m3x4((v >> 20) & 0xFu);
    hi.z = e4m3x4((v >> 24) & 0xFu);
    hi.w = e4m3x4(v >> 28);
}

__device__ __forceinline__ void store_e4m3_word(uint8_t *dst, uint32_t v)
{
    uint4 lo, hi;
    expand_e4m3_word(v, lo, hi);
    reinterpret_cast<uint4 *>(dst)[0] = lo;
    reinterpret_cast<uint4 *>(dst)[1] = hi;
}

// The same with streaming stores (evict first), for the helper warps of a Gram launch: the
// operands of the running product stay in L2.
__device__ __forceinline__ void store_e4m3_word_cs(uint8_t *dst, uint32_t v)
{
    uint4 lo, hi;
    expand_e4m3_word(v, lo, hi);
    __stcs(reinterpret_cast<uint4 *>(dst), lo);
    __stcs(reinterpret_cast<uint4 *>(dst) + 1, hi);
}

// x axis, straight from the packed store: a CTA stages both sublattices' words of 128
// consecutive rows (row = y + L z; four bundles B of 32 rows) in shared memory with coalesced
// loads; a warp then takes word column kw of both parity classes pi of those rows (lane = row
// in the bundle), transposes each 32 x 32 bit block in registers (five shuffle stages, each
// swapping the off-diagonal half-blocks of size j between lanes r and r ^ j), after which lane
// i holds, for site x = 2 (32 kw + i) + pi, the bits of the bundle's 32 rows.  The 64
// positions x = 64 kw .. 64 kw + 63 of the column are consecutive 128-byte lines of the chunk:
// the warp expands them into shared memory (16-byte piece c of position P at piece
// c ^ ((P >> 1) & 7), so both the scattered writes and the line-ordered reads are
// conflict-free) and writes the 8 KB with 512-byte coalesced stores.
__device__ __forceinline__ uint32_t transpose32_lane(uint32_t v, int lane)
{
    const uint32_t FULL = 0xffffffffu;
    const uint32_t lows[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const uint32_t low = lows[k];
        const uint32_t t = __shfl_xor_sync(FULL, v, j);
        v = (lane & j) ? ((v & ~low) | ((t & ~low) >> j)) : ((v & low) | ((t & low) << j));
    }
    return v;
}

static size_t expand_x_smem_bytes(int W) { return (size_t)128 * (2 * W + 1) * sizeof(uint32_t) + 8 * 64 * 128; }

__global__ void __launch_bounds__(256) k_expand_x_e4m3(const uint32_t *S0, const uint32_t *S1, Geom g, uint8_t *E)
{
    extern __shared__ __align__(16) uint32_t xt[];  // [128 rows][2 W + 1], then 8 warps x [64 lines][128 B]
    const int L = g.L, W = g.W, RS = 2 * W + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint4 *lines = reinterpret_cast<uint4 *>(xt + 128 * RS) + warp * 64 * 8;
    const int64_t nB4 = (int64_t)L * L / 128;  // chunks of 128 rows = 4 bundles of 32
    const int64_t blk = (int64_t)L * GT_KB;
    for (int64_t B4 = blockIdx.x; B4 < nB4; B4 += gridDim.x) {
        __syncthreads();  // the previous chunk's tile is consumed
        // coalesced: consecutive threads read consecutive words of the chunk's rows
        for (int e = tid; e < 128 * 2 * W; e += blockDim.x) {
            const int ri = e / (2 * W), c = e - ri * 2 * W;
            const int sub = c / W, kw = c - sub * W;
            xt[ri * RS + c] = __ldg((sub ? S1 : S0) + (128 * B4 + ri) * W + kw);
        }
        __syncthreads();
        for (int kw = warp; kw < W; kw += blockDim.x / 32) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int ri = 32 * b + lane;
                const uint32_t row = (uint32_t)(128 * B4 + ri);  // < L^2
                const uint32_t z = row / (uint32_t)L, y = row - z * (uint32_t)L;
#pragma unroll
                for (int pi = 0; pi < 2; ++pi) {
                    const uint32_t v = xt[ri * RS + (((pi + y + z) & 1u) ? W : 0) + kw];
                    uint4 lo, hi;
                    expand_e4m3_word(transpose32_lane(v, lane), lo, hi);
                    const int P = 2 * lane + pi, sw = lane & 7;  // (P >> 1) & 7
                    lines[P * 8 + ((2 * b) ^ sw)] = lo;
                    lines[P * 8 + ((2 * b + 1) ^ sw)] = hi;
                }
            }
            __syncwarp();
            uint4 *dst = reinterpret_cast<uint4 *>(E + B4 * blk + (int64_t)64 * kw * GT_KB);
#pragma unroll 4
            for (int j = 0; j < 16; ++j) {
                const int t = 32 * j + lane, P = t >> 3;
                dst[t] = lines[P * 8 + ((t & 7) ^ ((P >> 1) & 7))];
            }
            __syncwarp();
        }
    }
}

// y and z axes, one packed word each: column cc = (pi L + a) W + kw of position p (consecutive
// words of one lattice row), the 32 lines 32 cc .. 32 cc + 31.
__device__ __forceinline__ void expand_yz_word(const uint32_t *S0, const uint32_t *S1, const Geom &g, int axis,
                                               uint8_t *E, int p, int cc)
{
    const int L = g.L, W = g.W;
    const int64_t blk = (int64_t)L * GT_KB;  // bytes of one 128-line chunk of all positions
    const int kw = cc % W;
    const int rest = cc / W;  // pi L + a
    const int a = rest % L, pi = rest / L;
    const int y = axis == 1 ? p : a, z = axis == 1 ? a : p;
    const uint32_t v = __ldg((((pi + y + z) & 1) ? S1 : S0) + ((int64_t)z * L + y) * W + kw);
    store_e4m3_word(E + (int64_t)(cc >> 2) * blk + (int64_t)p * GT_KB + 32 * (cc & 3), v);
}

// The expansion a Gram launch's helper warps run for the next product: axis `axis` (1: y,
// 2: z) of the lattice (S0, S1) into E (nullptr: none).  (The x axis, bit-transposed, has a
// kernel of its own: run by the helper warps it slowed the product it shared the SMs with by
// more than its own 2.3 ms at L = 2048.)
struct ExpandJob {
    const uint32_t *S0, *S1;
    uint8_t *E;
    int axis;
};

// Helper thread h of nh: its share of job j.
__device__ __forceinline__ void run_expand_job(const ExpandJob &j, const Geom &g, int h, int nh)
{
    if (!j.E) return;
    // words i = h + nh (U m + u): the U loads of a round are issued before its stores
    constexpr int U = 16;
    const int L = g.L, W = g.W;
    const uint32_t ncols = (uint32_t)((int64_t)L * L / 32), total = (uint32_t)L * ncols;  // L^3 / 32 < 2^31
    const int64_t blk = (int64_t)L * GT_KB;
    for (uint32_t i0 = (uint32_t)h; i0 < total; i0 += (uint32_t)nh * U) {
        uint32_t v[U];
        uint8_t *dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + (uint32_t)nh * u;
            v[u] = 0;
            dst[u] = nullptr;
            if (i < total) {
                const int p = (int)(i / ncols), cc = (int)(i - (uint32_t)p * ncols);
                const int kw = cc % W, rest = cc / W;  // rest = pi L + a
                const int a = rest % L, pi = rest / L;
                const int y = j.axis == 1 ? p : a, z = j.axis == 1 ? a : p;
                v[u] = __ldg((((pi + y + z) & 1) ? j.S1 : j.S0) + ((int64_t)z * L + y) * W + kw);
                dst[u] = j.E + (int64_t)(cc >> 2) * blk + (int64_t)p * GT_KB + 32 * (cc & 3);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (dst[u]) store_e4m3_word_cs(dst[u], v[u]);
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int x, int y, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(mbar)
                 : "memory");
}

// One CTA per (tile bj, super-tile sb of columns 2 sb, 2 sb + 1, K slice), 2 sb + 1 >= bj: thread
// 0 loads the 128 x 128-byte box of tile bj and the 256 x 128-byte box of the super-tile by TMA
// (128-byte swizzle) into a ring of GT_STAGES stages, thread 32 issues four tcgen05.mma of
// 128 x 256 x 32 per stage into a 256-column fp32 accumulator in tensor memory and frees the
// stage by tcgen05.commit; then warps 0-3 read the accumulator and add each entry of an
// upper-triangle tile (bk >= bj, bk < nb) as -G/2 to D at its cyclic distance.  The CTAs of
// one K slice run together and stream the same columns, so L2 serves the tiles' repeated
// reads.  Warps 4-7 meanwhile expand the next product's axis (`next`) into the other scratch
// half; they wait on nothing and join the CTA at the barrier after the main loop.  Measured:
// L=1024 a whole measurement 2.18 ms against 2.93 with every expansion a kernel of its own;
// L=2048 21.1 against 21.5 ms (there the helpers' 8.6 GB of stores cost the product part of
// its L2 hits).
//
// Every wait is bounded (timeout_ns of %globaltimer).  A wait that gives up clears the CTA's
// `flag`, sets *err and the CTA stops without adding anything to D.  Before it leaves:
//  * the producer waits, bounded, on the `full` barrier of every stage whose TMA loads it
//    issued and the MMA thread did not consume, so that no bulk copy is still writing this
//    CTA's shared memory when the CTA exits (stages [mma_end, prod_end) of the ring);
//  * the MMA thread commits every MMA it issued to `done` and waits for it; only when that
//    commit has arrived is the tensor memory released.  If it has not (no MMA on resident
//    operands takes seconds, so this is not expected), the CTA records *err = 2 and skips
//    the dealloc rather than free tensor memory the tensor core may still write.
// No test provokes these paths; the stall test drops stage 0's loads of CTA 0 before any
// load or MMA is in flight.
__global__ void __launch_bounds__(GT_THREADS, 1) k_gram_tma(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB, int L, int nb,
                                                            int nunits, int split, int64_t *D, int *err,
                                                            uint64_t timeout_ns, int inject, ExpandJob next)
{
    extern __shared__ __align__(1024) uint8_t gsm[];
    uint8_t *stage0 = gsm;  // [S][A 16 KB, B 32 KB]
    long long *sacc = reinterpret_cast<long long *>(gsm + GT_STAGES * GT_STAGE_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(sacc + 1026);
    uint64_t *empty = full + GT_STAGES;
    uint64_t *done = empty + GT_STAGES;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(done + 1);
    int *flag = reinterpret_cast<int *>(tmem_holder + 1);
    int *mma_end = flag + 1;      // stages whose operands the MMA thread waited for
    int *mma_pending = flag + 2;  // 1: issued MMAs not known to be complete (keep the TMEM)

    const int H = L / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sl = blockIdx.x / nunits;
    int u = blockIdx.x - sl * nunits;
    const int nsb = (nb + 1) / 2;
    int bj = 0;
    while (u >= nsb - bj / 2) {
        u -= nsb - bj / 2;
        ++bj;
    }
    const int sb = bj / 2 + u;
    const int j0 = bj * TM_T, s0 = sb * GT_N;
    const int nk = (int)((int64_t)L * L / GT_KB);
    const int c0 = (int)((int64_t)nk * sl / split), c1 = (int)((int64_t)nk * (sl + 1) / split);
    const int n = c1 - c0;

    for (int i = tid; i <= H; i += GT_THREADS) sacc[i] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(GT_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < GT_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *flag = 1;
        *mma_end = 0;
        *mma_pending = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    int prod_end = 0;  // producer: stages [0, prod_end) were armed (expect_tx) and loaded
    if (warp >= 4) {  // helper warps: the next product's expansion, into the other scratch half
        run_expand_job(next, make_geom(L), (int)(blockIdx.x * (GT_THREADS - 128) + tid - 128),
                       (int)(gridDim.x * (GT_THREADS - 128)));
    } else if (tid == 0) {  // producer
        for (int t = 0; t < n; ++t) {
            const int st = t % GT_STAGES;
            if (t >= GT_STAGES &&
                !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((t / GT_STAGES) - 1) & 1), timeout_ns)) {
                *flag = 0;
                break;
            }
            if (!*(volatile int *)flag) break;
            const uint32_t sa = smem_u32(stage0 + st * GT_STAGE_BYTES);
            mbar_expect_tx(smem_u32(&full[st]), GT_STAGE_BYTES);
            prod_end = t + 1;
            if (inject && blockIdx.x == 0 && t == 0) continue;  // test hook: this stage never fills
            tma_load_2d(sa, &tmA, 0, (c0 + t) * L + j0, smem_u32(&full[st]));
            tma_load_2d(sa + TM_T * GT_KB, &tmB, 0, (c0 + t) * L + s0, smem_u32(&full[st]));
        }
    } else if (tid == 32) {  // MMA issuer
        int t = 0;
        for (; t < n; ++t) {
            const int st = t % GT_STAGES;
            if (!*(volatile int *)flag) break;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((t / GT_STAGES) & 1), timeout_ns)) {
                *flag = 0;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(stage0 + st * GT_STAGE_BYTES);
#pragma unroll
            for (int q = 0; q < GT_KB / 32; ++q) {
                const uint64_t ad = umma_desc_sw128(sa + 32 * q), bd = umma_desc_sw128(sa + TM_T * GT_KB + 32 * q);
                const uint32_t acc = (t > 0 || q > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(UMMA_IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[st])));
        }
        *mma_end = t;
        if (t > 0) {  // the last commit covers every MMA before it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(done)));
            if (!mbar_wait(smem_u32(done), 0u, timeout_ns)) {
                *flag = 0;
                // one more bounded window before the tensor memory is declared still in use
                if (!mbar_wait(smem_u32(done), 0u, timeout_ns)) *mma_pending = 1;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && !*flag) {
        // drain: every stage armed and loaded but not consumed by the MMA thread lands
        // before the CTA may leave (at most GT_STAGES of them, all distinct ring slots)
        for (int t = *mma_end; t < prod_end; ++t) {
            if (inject && blockIdx.x == 0 && t == 0) continue;  // no load was issued for it
            if (!mbar_wait(smem_u32(&full[t % GT_STAGES]), (uint32_t)((t / GT_STAGES) & 1), timeout_ns))
                atomicExch(err, 3);
        }
    }
    __syncthreads();
    const bool ok = *flag && n > 0;
    if (ok && warp < 4) {  // warp w reads tensor-memory lanes 32 w .. 32 w + 31
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int j = j0 + 32 * warp + lane;  // this thread's row of the tile (TMEM lane)
#pragma unroll 1
        for (int cc = 0; cc < GT_N; cc += 16) {
            const int bk = 2 * sb + cc / TM_T;
            if (bk < bj || bk >= nb) continue;  // lower-triangle or missing tile of the super-tile
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = s0 + cc + q;
                const long long G = (long long)__float2int_rn(__uint_as_float(v[q]));
                if (bj == bk) {
                    int d = k - j;
                    if (d < 0) d += L;
                    if (d >= 1 && d <= H) atomicAdd((unsigned long long *)&sacc[d], (unsigned long long)G);
                } else {
                    const int d = k - j;  // 0 < d < L
                    if (d <= H) atomicAdd((unsigned long long *)&sacc[d], (unsigned long long)G);
                    if (L - d <= H) atomicAdd((unsigned long long *)&sacc[L - d], (unsigned long long)G);
                }
            }
        }
    }
    if (!*flag && tid == 0) atomicCAS(err, 0, 1);
    if (*mma_pending && tid == 0) atomicExch(err, 2);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && !*mma_pending)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_N));
    if (!ok) return;
    for (int i = 1 + tid; i <= H; i += GT_THREADS)
        if (sacc[i]) atomicAdd((unsigned long long *)(D + i), (unsigned long long)(-(sacc[i] / 2)));
}

static size_t gram_smem_bytes() { return (size_t)GT_STAGES * GT_STAGE_BYTES + 1026 * 8 + (2 * GT_STAGES + 1) * 8 + 32; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        looked = true;
    }
    return fn;
}

bool corr_mma_supported(int L) { return L >= 256 && L <= 2048 && L % TM_T == 0 && L % 64 == 0; }

size_t corr_mma_scratch_bytes(int L, int R)
{
    (void)R;  // replicas are multiplied one after the other through two expanded axes
    return (size_t)2 * L * L * L;
}

cudaError_t launch_corr_mma(const uint32_t *lat, int L, int R, int64_t *rec, uint32_t *scratch, int *err,
                            cudaStream_t s, int64_t *launches, double timeout_s, int inject)
{
    const uint64_t timeout_ns = (uint64_t)(timeout_s * 1e9);
    const Geom g = make_geom(L);
    // two halves of L^3 bytes: product i reads half i % 2 while its helper warps expand product
    // i + 1 into the other
    uint8_t *E[2] = {reinterpret_cast<uint8_t *>(scratch), reinterpret_cast<uint8_t *>(scratch) + (size_t)L * L * L};
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // E viewed as rows of 128 bytes: row (chunk * L + position); boxes of 128 and 256 rows
    CUtensorMap tmA[2], tmB[2];
    const cuuint64_t gdim[2] = {(cuuint64_t)GT_KB, (cuuint64_t)L * L * L / GT_KB};
    const cuuint64_t gstride[1] = {(cuuint64_t)GT_KB};
    const cuuint32_t boxA[2] = {GT_KB, TM_T}, boxB[2] = {GT_KB, GT_N};
    const cuuint32_t estr[2] = {1, 1};
    for (int h = 0; h < 2; ++h)
        if (enc(&tmA[h], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, E[h], gdim, gstride, boxA, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
            enc(&tmB[h], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, E[h], gdim, gstride, boxB, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const size_t smem = gram_smem_bytes();
    if ((e = cudaFuncSetAttribute(k_gram_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    const int nb = L / TM_T, nsb = (nb + 1) / 2;
    int nunits = 0;  // (tile row bj, super-tile sb >= bj / 2)
    for (int bj = 0; bj < nb; ++bj) nunits += nsb - bj / 2;
    int split = sms / nunits;  // one CTA per SM: K slices x units <= SMs
    if (split < 1) split = 1;
    const int64_t H = L / 2, RL = 3 + 3 * (H + 1);
    const size_t xsm = expand_x_smem_bytes(g.W);
    if ((e = cudaFuncSetAttribute(k_expand_x_e4m3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm)) !=
        cudaSuccess)
        return e;
    // per replica: x expanded by its own kernel into half 0; its product's helper warps expand
    // y into half 1, and the y product's helpers z into half 0; the z product runs alone
    for (int r = 0; r < R; ++r) {
        const uint32_t *S0 = lat + 2 * (int64_t)r * g.nw, *S1 = S0 + g.nw;
        k_expand_x_e4m3<<<(unsigned)std::min<int64_t>((int64_t)L * L / 128, (int64_t)sms * 2), 256, xsm, s>>>(
            S0, S1, g, E[0]);
        for (int axis = 0; axis < 3; ++axis) {
            const ExpandJob next = axis < 2 ? ExpandJob{S0, S1, E[(axis + 1) % 2], axis + 1}
                                            : ExpandJob{nullptr, nullptr, nullptr, 0};
            k_gram_tma<<<(unsigned)(nunits * split), GT_THREADS, smem, s>>>(
                tmA[axis % 2], tmB[axis % 2], L, nb, nunits, split, rec + r * RL + 3 + axis * (H + 1), err,
                timeout_ns, inject && r == 0 && axis == 1, next);
        }
    }
    if (launches) *launches += 4 * (int64_t)R;
    return cudaGetLastError();
}

}  // namespace ising
