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
// off-diagonal tile stands for both ordered pairs (j, k) and (k, j).  The 128 x 128 tiles are
// accumulated by tcgen05.mma in tensor memory (kernel below); each entry's -G/2 is added to D
// at its cyclic distance; the records start from N/2.
#include "common.cuh"
#include "kernels.h"

namespace ising {

constexpr int TM_T = 128;        // positions per tile side (M = N = 128)
constexpr int UM_NP = 8;         // columns (K = 32 lines each) per panel, a multiple of 4
constexpr int UM_PD = 6;         // packed panels in flight (ring slots)
constexpr int TM_THREADS = 256;  // 8 warps: staging and expansion; warp w reads TMEM lane quarter w % 4
constexpr int UMMA_WAIT_LIMIT = 1 << 22;  // try_wait rounds before a wait gives up

// x-axis columns: bundle B = rows 32B .. 32B+31 (row = y + L z); XT[B*L + x] has bit i =
// spin (x, row 32B + i) (1 = up).  One warp per (bundle, x-parity, word): 32 ballots.
__global__ void k_transpose_x(const uint32_t *lat, Geom g, uint32_t *XT)
{
    const int r = blockIdx.y;
    const uint32_t *S0 = lat + 2 * (int64_t)r * g.nw;
    const uint32_t *S1 = S0 + g.nw;
    const int L = g.L, W = g.W;
    const int64_t nB = (int64_t)L * L / 32;
    uint32_t *X = XT + (int64_t)r * nB * L;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t task = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); task < nB * 2 * W;
         task += nwarps) {
        const int64_t B = task / (2 * W);
        const int rem = (int)(task - B * 2 * W);
        const int pi = rem / W, kw = rem - pi * W;
        const int64_t row = 32 * B + lane;
        const int y = (int)(row % L), z = (int)(row / L);
        const uint32_t v = (((pi + y + z) & 1) ? S1 : S0)[row * W + kw];
        uint32_t mine = 0u;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const unsigned bal = __ballot_sync(0xffffffffu, (v >> k) & 1u);
            if (lane == k) mine = bal;
        }
        X[B * L + 2 * (32 * kw + lane) + pi] = mine;
    }
}

// Four e4m3 values from the four bits of n (n < 16): bit i -> byte i, +1.0 (0x38) when
// set, -1.0 (0xB8) when clear.  The multiplier places bit i at bit 8i + 7 (and the other
// bits of n at positions that the mask drops, without carries).
__device__ __forceinline__ uint32_t e4m3x4(uint32_t n)
{
    return ((n * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u;
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
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

// Instruction descriptor: D in f32, A and B e4m3, both K-major, M = 128, N = 128.
constexpr uint32_t UMMA_IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TM_T >> 3) << 17) |
                                ((uint32_t)(TM_T >> 4) << 24);

// Bounded wait for phase `parity` of an mbarrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (int it = 0; it < UMMA_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Work of one replica: the three axes x npairs tile pairs (bj <= bk) x npan panels of NP
// columns (K = 32 lines each).  Persistent CTAs take equal contiguous shares of that list; a
// share is cut into segments that stay within one tile pair, each accumulated in a
// 128-column fp32 tile of tensor memory and then added to S(r) of its axis.
//
// Per panel the packed words (staged by cp.async, two panels ahead) are expanded by all
// threads into e4m3 operands in K-major 128-byte swizzled atoms (the swizzle keeps both the
// expansion's stores and the tensor core's reads free of bank conflicts), and one thread
// issues NP tcgen05.mma; tcgen05.commit on the stage's mbarrier frees
// the operand stage for the panel after next.  Waits are made by thread 0 and shared through
// the block, so every thread takes the same path; a wait that gives up sets *err and the CTA
// stops after releasing its tensor memory.
template <int NP, int PD>
__global__ void __launch_bounds__(TM_THREADS, 1) k_corr_umma(const uint32_t *lat, const uint32_t *XT, Geom g, int nb,
                                                              int npairs, int64_t *rec, int *err)
{
    extern __shared__ __align__(1024) uint8_t usm[];
    uint8_t *op = usm;  // [2 stages][A, B][NP/4 column groups][16 atoms of 8 rows x 128 B]
    uint32_t *panel = reinterpret_cast<uint32_t *>(usm + 2 * NP * 2 * 4096);       // [PD][NP][256]
    long long *sacc = reinterpret_cast<long long *>(panel + PD * NP * 2 * TM_T);   // S(r), r <= L/2
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sacc + 1026);                    // [2]
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mbar + 2);
    int *flag = reinterpret_cast<int *>(tmem_holder + 1);

    const int r = blockIdx.y;
    const int L = g.L, H = L / 2, W = g.W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t *S0 = lat + 2 * (int64_t)r * g.nw;
    const uint32_t *S1 = S0 + g.nw;
    const int64_t ncols = 2 * (int64_t)L * W;  // columns per axis (x: L^2/32 bundles, the same count)
    const int64_t npan = ncols / NP;
    const int64_t total = 3LL * npairs * npan;
    const int64_t w_begin = total * blockIdx.x / gridDim.x, w_end = total * (blockIdx.x + 1) / gridDim.x;

    for (int i = tid; i <= H; i += TM_THREADS) sacc[i] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TM_T));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    int gi = 0;  // panels processed by this CTA: selects the stage and the mbarrier phase
    for (int64_t w = w_begin; w < w_end;) {
        const int64_t unit = w / npan;  // (axis, pair)
        const int64_t pan0 = w - unit * npan;
        const int64_t pan1 = (w_end - w) < (npan - pan0) ? pan0 + (w_end - w) : npan;
        const int n = (int)(pan1 - pan0);
        w += n;
        const int axis = (int)(unit / npairs);
        int p = (int)(unit - (int64_t)axis * npairs);
        int bj = 0;
        while (p >= nb - bj) {
            p -= nb - bj;
            ++bj;
        }
        const int bk = bj + p;
        const int j0 = bj * TM_T, k0 = bk * TM_T;
        const uint32_t *X = axis == 0 ? XT + (int64_t)r * ncols * L : nullptr;

        // staging: element (c, pp) of a panel = column c, pair position pp (pp < 128: tile bj
        // (A), else tile bk (B)); the threads take consecutive elements
        auto issue = [&](int64_t pan, int stage) {
            uint32_t *pl = panel + stage * NP * 2 * TM_T;
            if (axis == 0) {  // XT rows are contiguous in position: consecutive pp
#pragma unroll
                for (int idx = tid; idx < NP * 2 * TM_T; idx += TM_THREADS) {
                    const int c = idx / (2 * TM_T), pp = idx % (2 * TM_T);
                    const int jj = pp < TM_T ? j0 + pp : k0 + (pp - TM_T);
                    cp_async4(&pl[c * 2 * TM_T + pp], X + (pan * NP + c) * (int64_t)L + jj);
                }
            } else {
                // consecutive threads take consecutive columns of one position: consecutive
                // words of one row (coalesced); the thread's column is fixed
                const int c = tid % NP;
                const int cc = (int)(pan * NP) + c;
                const int pi = cc / (L * W);
                const int rem = cc - pi * L * W;
                const int a = rem / W;
                const int kw = rem - a * W;
#pragma unroll
                for (int idx = tid; idx < NP * 2 * TM_T; idx += TM_THREADS) {
                    const int pp = idx / NP;
                    const int jj = pp < TM_T ? j0 + pp : k0 + (pp - TM_T);
                    const int y = axis == 1 ? jj : a, z = axis == 1 ? a : jj;
                    cp_async4(&pl[c * 2 * TM_T + pp], (((pi + y + z) & 1) ? S1 : S0) + ((int64_t)z * L + y) * W + kw);
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };

        // packed panels run PD ahead in a ring of their own (panel i of the segment in slot
        // (gi0 + i) % PD); operand stages alternate with gi
        const int gi0 = gi;
        for (int k = 0; k < PD - 1 && k < n; ++k) issue(pan0 + k, (gi0 + k) % PD);
        for (int i = 0; i < n; ++i, ++gi) {
            const int st = gi & 1;
            if (i + PD - 1 < n) issue(pan0 + i + PD - 1, (gi0 + i + PD - 1) % PD);
            if (i + PD - 1 < n)
                asm volatile("cp.async.wait_group %0;\n" ::"n"(PD - 1) : "memory");
            else
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            if (gi >= 2 && tid == 0 && !mbar_wait(smem_u32(&mbar[st]), (uint32_t)(((gi - 2) >> 1) & 1))) *flag = 0;
            __syncthreads();  // packed panel visible; operand stage st free (or the wait gave up)
            if (!*flag) break;
            const uint32_t *pl = panel + ((gi0 + i) % PD) * NP * 2 * TM_T;
            uint8_t *ops = op + st * NP * 2 * 4096;
#pragma unroll
            for (int idx = tid; idx < NP * 2 * TM_T; idx += TM_THREADS) {
                const int c = idx / (2 * TM_T), pp = idx % (2 * TM_T);
                const int pos = pp & (TM_T - 1), half = pp >> 7;
                const uint32_t v = pl[c * 2 * TM_T + pp];
                uint4 lo, hi;
                lo.x = e4m3x4(v & 0xFu);
                lo.y = e4m3x4((v >> 4) & 0xFu);
                lo.z = e4m3x4((v >> 8) & 0xFu);
                lo.w = e4m3x4((v >> 12) & 0xFu);
                hi.x = e4m3x4((v >> 16) & 0xFu);
                hi.y = e4m3x4((v >> 20) & 0xFu);
                hi.z = e4m3x4((v >> 24) & 0xFu);
                hi.w = e4m3x4(v >> 28);
                // operand (half) of column group c/4: atom pos/8, row r = pos%8; the column's
                // two 16-byte chunks 2(c%4) and 2(c%4)+1 of the row, swizzled by r
                const int r8 = pos & 7, ch = 2 * (c & 3);
                uint8_t *row = ops + (half * (NP / 4) + (c >> 2)) * 16384 + (pos >> 3) * 1024 + r8 * 128;
                *reinterpret_cast<uint4 *>(row + ((ch ^ r8) << 4)) = lo;        // lines 0..15 of the column
                *reinterpret_cast<uint4 *>(row + (((ch + 1) ^ r8) << 4)) = hi;  // lines 16..31
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();  // operands written; packed panel consumed
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int c = 0; c < NP; ++c) {
                    const uint32_t koff = (uint32_t)((c >> 2) * 16384 + (c & 3) * 32);
                    const uint64_t ad = umma_desc_sw128(smem_u32(ops) + koff);
                    const uint64_t bd = umma_desc_sw128(smem_u32(ops) + (NP / 4) * 16384 + koff);
                    const uint32_t acc = (i > 0 || c > 0) ? 1u : 0u;
                    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                 "l"(ad), "l"(bd), "r"(UMMA_IDESC), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[st])));
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        // the segment's last commit covers every MMA issued before it
        if (tid == 0 && *flag && !mbar_wait(smem_u32(&mbar[(gi - 1) & 1]), (uint32_t)(((gi - 1) >> 1) & 1)))
            *flag = 0;
        __syncthreads();
        if (!*flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3;            // TMEM lanes this warp may read
        const int j = j0 + 32 * quarter + lane;  // this thread's row of the tile
        constexpr int CPW = TM_T / (TM_THREADS / 128);  // accumulator columns per warp
#pragma unroll 1
        for (int c0 = (warp >> 2) * CPW; c0 < (warp >> 2) * CPW + CPW; c0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = k0 + c0 + q;
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
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the accumulator is read; the next segment may overwrite it
        int64_t *D = rec + (int64_t)r * (3 + 3 * (int64_t)(H + 1)) + 3 + (int64_t)axis * (H + 1);
        for (int i = 1 + tid; i <= H; i += TM_THREADS)
            if (sacc[i]) {
                atomicAdd((unsigned long long *)(D + i), (unsigned long long)(-(sacc[i] / 2)));
                sacc[i] = 0;
            }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!*flag && tid == 0) {
        atomicExch(err, 1);
        if (gi > 0) mbar_wait(smem_u32(&mbar[(gi - 1) & 1]), (uint32_t)(((gi - 1) >> 1) & 1));  // in-flight MMAs
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_T));
}

template <int NP, int PD>
static size_t umma_smem_bytes()
{
    return (size_t)2 * NP * 2 * 4096 + (size_t)PD * NP * 2 * TM_T * 4 + 1026 * 8 + 2 * 8 + 8;
}

bool corr_mma_supported(int L) { return L >= 256 && L <= 2048 && L % TM_T == 0 && L % 64 == 0; }

cudaError_t launch_corr_mma(const uint32_t *lat, int L, int R, int64_t *rec, uint32_t *xt_scratch, int *err,
                            cudaStream_t s, int64_t *launches)
{
    const Geom g = make_geom(L);
    {
        const int64_t tasks = (int64_t)L * L / 32 * 2 * g.W;
        int64_t blocks = (tasks + 7) / 8;
        if (blocks > 152 * 32) blocks = 152 * 32;
        k_transpose_x<<<dim3((unsigned)blocks, (unsigned)R), 256, 0, s>>>(lat, g, xt_scratch);
    }
    constexpr int NP = UM_NP, PD = UM_PD;
    const int nb = L / TM_T;
    const int npairs = nb * (nb + 1) / 2;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const size_t smem = umma_smem_bytes<NP, PD>();
    if ((e = cudaFuncSetAttribute(k_corr_umma<NP, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    int occ = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_corr_umma<NP, PD>, TM_THREADS, smem)) != cudaSuccess)
        return e;
    if (occ < 1) occ = 1;
    // persistent: one wave of CTAs shares the replicas' work equally
    int ctas = (int)(((int64_t)occ * sms + R - 1) / R);
    if (ctas < 1) ctas = 1;
    k_corr_umma<NP, PD><<<dim3((unsigned)ctas, (unsigned)R), TM_THREADS, smem, s>>>(lat, xt_scratch, g, nb, npairs, rec,
                                                                                err);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace ising
