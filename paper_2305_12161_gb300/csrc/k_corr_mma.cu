// Axis correlation sums D_a(r) on the tensor cores.
//
// Along one axis the lattice is L^2 lines of L sites.  With s = +-1,
//   sum_i [s_i != s_(i + r e_a)] = (L * L^2 - S(r)) / 2,   S(r) = sum_j G[j][(j + r) mod L],
// where G[j][k] = sum over lines of s(j) s(k) is the Gram matrix of the L positions over
// the lines: a dense contraction of length L^2.  A packed word holds the same position of
// 32 lines, so one word is the K = 32 slice of one m16n8k32 fp8 MMA: its bits become e4m3
// values +1 / -1 (exact), products accumulate in fp32, and every partial sum is an even
// integer of magnitude <= L^2 <= 2^24, so the result is exact.
//
// Only the upper block triangle of G is computed (G is symmetric); an entry of an
// off-diagonal tile stands for both ordered pairs (j, k) and (k, j).  CTA = 128 x 128 tile
// of G (4 warps of 64 x 64) over a range of columns (split over K); columns stream through
// a two-stage shared-memory panel by cp.async.  Each entry's -G/2 is added to D at its
// cyclic distance; the records start from N/2.
#include "common.cuh"
#include "kernels.h"

namespace ising {

constexpr int TM_T = 128;       // positions per tile side
constexpr int TM_NP = 16;       // columns per staged panel
constexpr int TM_THREADS = 128;  // 4 warps, 2 x 2 warp tiles of 64 x 64

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

__device__ __forceinline__ void mma_e4m3(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(TM_THREADS, 2) k_corr_mma(const uint32_t *lat, const uint32_t *XT, Geom g,
                                                             int nb, int split, int64_t *rec)
{
    __shared__ __align__(16) uint32_t panel[2][TM_NP][2 * TM_T];  // [stage][column][position]
    __shared__ long long sacc[2048 / 2 + 1];                       // S(r) of this CTA, r <= L/2 (L <= 2048)
    const int axis = blockIdx.z, r = blockIdx.y;
    const int L = g.L, H = L / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;  // MMA fragment group and thread-in-group
    const int wm = warp >> 1, wn = warp & 1;
    // tile pair (bj <= bk) and K range of this CTA
    int p = blockIdx.x / split;
    const int s = blockIdx.x - p * split;
    int bj = 0;
    while (p >= nb - bj) {
        p -= nb - bj;
        ++bj;
    }
    const int bk = bj + p;
    const int j0 = bj * TM_T, k0 = bk * TM_T;
    const uint32_t *S0 = lat + 2 * (int64_t)r * g.nw;
    const uint32_t *S1 = S0 + g.nw;
    const int64_t ncols = axis == 0 ? (int64_t)L * L / 32 : 2 * (int64_t)L * g.W;
    const uint32_t *X = axis == 0 ? XT + (int64_t)r * ncols * L : nullptr;
    const int64_t npan = ncols / TM_NP;
    const int64_t pan0 = npan * s / split, pan1 = npan * (s + 1) / split;
    for (int i = tid; i <= H; i += TM_THREADS) sacc[i] = 0;

    // Staging: x axis — thread copies positions tid and tid+128 of columns 0..15 (XT rows
    // are contiguous in position); y/z axes — thread copies column (tid & 15) at positions
    // (tid >> 4) + 8i, i < 32 (consecutive columns are consecutive words).  Address math is
    // done once per panel.
    const int L_ = L, W = g.W;
    auto issue = [&](int64_t pan, int stage) {
        if (axis == 0) {
            const uint32_t *base = X + pan * TM_NP * (int64_t)L_;
#pragma unroll 4
            for (int i = 0; i < 2 * TM_NP; ++i) {
                const int pp = tid + TM_T * (i & 1);
                const int c = i >> 1;
                const int j = pp < TM_T ? j0 + pp : k0 + (pp - TM_T);
                cp_async4(&panel[stage][c][pp], base + (int64_t)c * L_ + j);
            }
        } else {
            const int cc = tid & (TM_NP - 1);
            const int c = (int)(pan * TM_NP) + cc;
            const int pi = c / (L_ * W);
            const int rem = c - pi * L_ * W;
            const int a = rem / W;
            const int kw = rem - a * W;
#pragma unroll 4
            for (int i = 0; i < 2 * TM_T / (TM_THREADS / TM_NP); ++i) {
                const int pp = (tid >> 4) + (TM_THREADS / TM_NP) * i;
                const int j = pp < TM_T ? j0 + pp : k0 + (pp - TM_T);
                const int y = axis == 1 ? j : a, z = axis == 1 ? a : j;
                const uint32_t *src = (((pi + y + z) & 1) ? S1 : S0) + ((int64_t)z * L_ + y) * W + kw;
                cp_async4(&panel[stage][cc][pp], src);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    float acc[4][8][4];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int h = 0; h < 8; ++h)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[f][h][v] = 0.f;

    if (pan0 < pan1) issue(pan0, 0);
    for (int64_t pan = pan0; pan < pan1; ++pan) {
        const int cur = (int)((pan - pan0) & 1);
        if (pan + 1 < pan1) {
            issue(pan + 1, cur ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < TM_NP; ++c) {
            const uint32_t *col = panel[cur][c];
            uint32_t a[4][4], b[4][2];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const uint32_t w0 = col[64 * wm + 16 * f + gq] >> (4 * tq);
                const uint32_t w1 = col[64 * wm + 16 * f + gq + 8] >> (4 * tq);
                a[f][0] = e4m3x4(w0 & 0xFu);          // row g,   k = 4t .. 4t+3
                a[f][1] = e4m3x4(w1 & 0xFu);          // row g+8, k = 4t .. 4t+3
                a[f][2] = e4m3x4((w0 >> 16) & 0xFu);  // row g,   k = 16+4t ..
                a[f][3] = e4m3x4((w1 >> 16) & 0xFu);  // row g+8, k = 16+4t ..
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {  // B fragments in two halves (register pressure)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t w = col[TM_T + 64 * wn + 8 * (4 * hh + h) + gq] >> (4 * tq);
                    b[h][0] = e4m3x4(w & 0xFu);          // column g, k = 4t ..
                    b[h][1] = e4m3x4((w >> 16) & 0xFu);  // column g, k = 16+4t ..
                }
#pragma unroll
                for (int f = 0; f < 4; ++f)
#pragma unroll
                    for (int h = 0; h < 4; ++h) mma_e4m3(acc[f][4 * hh + h], a[f], b[h]);
            }
        }
        __syncthreads();  // the stage is refilled by the next-but-one issue
    }

    // epilogue: add each entry to S at its cyclic distance
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int h = 0; h < 8; ++h)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = j0 + 64 * wm + 16 * f + gq + (v >> 1) * 8;
                const int k = k0 + 64 * wn + 8 * h + 2 * tq + (v & 1);
                const long long G = (long long)__float2int_rn(acc[f][h][v]);
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
    __syncthreads();
    int64_t *D = rec + (int64_t)r * (3 + 3 * (int64_t)(H + 1)) + 3 + (int64_t)axis * (H + 1);
    for (int i = 1 + tid; i <= H; i += TM_THREADS)
        if (sacc[i]) atomicAdd((unsigned long long *)(D + i), (unsigned long long)(-(sacc[i] / 2)));
}

bool corr_mma_supported(int L) { return L >= 256 && L <= 2048 && L % TM_T == 0 && L % 64 == 0; }

cudaError_t launch_corr_mma(const uint32_t *lat, int L, int R, int64_t *rec, uint32_t *xt_scratch, cudaStream_t s,
                            int64_t *launches)
{
    const Geom g = make_geom(L);
    {
        const int64_t tasks = (int64_t)L * L / 32 * 2 * g.W;
        int64_t blocks = (tasks + 7) / 8;
        if (blocks > 152 * 32) blocks = 152 * 32;
        k_transpose_x<<<dim3((unsigned)blocks, (unsigned)R), 256, 0, s>>>(lat, g, xt_scratch);
    }
    const int nb = L / TM_T;
    const int npairs = nb * (nb + 1) / 2;
    const int64_t npan = (2 * (int64_t)L * g.W) / TM_NP;  // equal for the three axes
    int split = (int)((8LL * 304) / (3LL * npairs * R));
    if (split < 1) split = 1;
    if (split > npan) split = (int)npan;
    k_corr_mma<<<dim3((unsigned)(npairs * split), (unsigned)R, 3), TM_THREADS, 0, s>>>(lat, xt_scratch, g, nb, split,
                                                                                      rec);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace ising
