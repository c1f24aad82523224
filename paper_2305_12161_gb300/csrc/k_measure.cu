// Measurement kernels on the packed store (Eq. (2) and the energy of H = -sum s_i s_j):
//   M = sum_i s_i, B = #unequal nearest-neighbour pairs, and the axis correlation sums
//   D_a(r) = #{ i : s_i != s_(i + r e_a) }, a in {x,y,z}, r = 0..L/2, as int64.
//
// Every bond joins an even and an odd site, so B is the sum over sublattice-0 words of
// popc(s ^ neighbour) for its six neighbour words.
//
// D_a(r) is computed on "columns": sequences of L words whose 32 bit lanes are 32
// independent lines of sites along axis a.  For a line parity class pi (sites
// x = 2k + pi) the word of row (y,z) is V_pi(y,z) = sublattice ((pi + y + z) mod 2) at
// that row, so along y or z the words of one (kw, pi) and the other coordinate form a
// column directly.  Along x, bundles of 32 rows are bit-transposed (warp ballots) into a
// column T[x] whose lane b is row b of the bundle.  Then, per column,
//   D_a(r) += sum_j popc(col[j] ^ col[(j + r) mod L]),
// staged in shared memory (extended by L/2 words so that j + r never wraps).
#include "common.cuh"
#include "kernels.h"

namespace ising {

__device__ __forceinline__ int64_t rec_len(int L) { return 3 + 3 * (int64_t)(L / 2 + 1); }

// corr: 0 = correlations not measured (-1), 1 = summed from 0, 2 = tensor-core path,
// which subtracts from N/2 (D_a(0) stays 0).
__global__ void k_rec_init(int64_t *rec, int L, int R, int64_t t, int corr)
{
    const int64_t RL = rec_len(L);
    const int64_t H1 = L / 2 + 1;
    const int64_t half_n = (int64_t)L * L * L / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < RL * R; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i % RL;
        int64_t v;
        if (j == 0) v = t;
        else if (j < 3) v = 0;
        else if (corr == 0) v = -1;
        else if (corr == 2 && (j - 3) % H1 != 0) v = half_n;
        else v = 0;
        rec[i] = v;
    }
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// M and B of replica blockIdx.y.
__global__ void k_mb(const uint32_t *lat, Geom g, int64_t *rec)
{
    const int r = blockIdx.y;
    const uint32_t *S0 = lat + (2 * (int64_t)r) * g.nw;
    const uint32_t *S1 = S0 + g.nw;
    long long m = 0, b = 0;
    for (int64_t sw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sw < g.nw; sw += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = __ldg(S0 + sw);
        const Nbrs n = load_nbrs(S1, g, sw, 0);
        b += __popc(s ^ n.C) + __popc(s ^ n.X) + __popc(s ^ n.Ym) + __popc(s ^ n.Yp) + __popc(s ^ n.Zm) +
             __popc(s ^ n.Zp);
        m += 2 * (__popc(s) + __popc(n.C)) - 2 * g.RB;
    }
    __shared__ long long red[2][32];
    m = warp_sum(m);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = m;
        red[1][wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        m = lane < nw ? red[0][lane] : 0;
        b = lane < nw ? red[1][lane] : 0;
        m = warp_sum(m);
        b = warp_sum(b);
        if (lane == 0) {
            const int64_t RL = rec_len(g.L);
            atomicAdd(reinterpret_cast<unsigned long long *>(rec + r * RL + 1), (unsigned long long)m);
            atomicAdd(reinterpret_cast<unsigned long long *>(rec + r * RL + 2), (unsigned long long)b);
        }
    }
}

// The same counts for L a multiple of 256: one thread per uint4 of sublattice 0 (128 sites of
// one row), rows found with 32-bit divisions (L^3 / 256 < 2^32) instead of 64-bit ones.
__global__ void k_mb4(const uint32_t *lat, Geom g, int64_t *rec)
{
    const int r = blockIdx.y;
    const uint4 *S0 = reinterpret_cast<const uint4 *>(lat + (2 * (int64_t)r) * g.nw);
    const uint4 *S1 = S0 + g.nw / 4;
    const uint32_t L = (uint32_t)g.L, W4 = L / 256, n4 = (uint32_t)(g.nw / 4);
    long long m = 0, b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
        const uint32_t row = i / W4, cx = i - row * W4;
        const uint32_t z = row / L, y = row - z * L;
        const uint4 s = __ldg(S0 + i);
        const uint4 C = __ldg(S1 + i);
        // x-neighbours that are not C itself: shifted by one site towards x - 1 (p = 0) or x + 1
        uint4 X;
        if (((y + z) & 1u) == 0) {
            const uint32_t e = __ldg(reinterpret_cast<const uint32_t *>(S1 + row * W4 + (cx == 0 ? W4 - 1 : cx - 1)) + 3);
            X = make_uint4((C.x << 1) | (e >> 31), (C.y << 1) | (C.x >> 31), (C.z << 1) | (C.y >> 31),
                           (C.w << 1) | (C.z >> 31));
        } else {
            const uint32_t e = __ldg(reinterpret_cast<const uint32_t *>(S1 + row * W4 + (cx == W4 - 1 ? 0 : cx + 1)));
            X = make_uint4((C.x >> 1) | (C.y << 31), (C.y >> 1) | (C.z << 31), (C.z >> 1) | (C.w << 31),
                           (C.w >> 1) | (e << 31));
        }
        const uint32_t ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
        const uint32_t zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
        const uint4 Ym = __ldg(S1 + (z * L + ym) * W4 + cx), Yp = __ldg(S1 + (z * L + yp) * W4 + cx);
        const uint4 Zm = __ldg(S1 + (zm * L + y) * W4 + cx), Zp = __ldg(S1 + (zp * L + y) * W4 + cx);
        auto bonds = [&](uint32_t sw, uint32_t c, uint32_t x, uint32_t a, uint32_t bb, uint32_t d, uint32_t e) {
            return __popc(sw ^ c) + __popc(sw ^ x) + __popc(sw ^ a) + __popc(sw ^ bb) + __popc(sw ^ d) + __popc(sw ^ e);
        };
        b += bonds(s.x, C.x, X.x, Ym.x, Yp.x, Zm.x, Zp.x) + bonds(s.y, C.y, X.y, Ym.y, Yp.y, Zm.y, Zp.y) +
             bonds(s.z, C.z, X.z, Ym.z, Yp.z, Zm.z, Zp.z) + bonds(s.w, C.w, X.w, Ym.w, Yp.w, Zm.w, Zp.w);
        m += 2 * (__popc(s.x) + __popc(s.y) + __popc(s.z) + __popc(s.w) + __popc(C.x) + __popc(C.y) + __popc(C.z) +
                  __popc(C.w)) -
             2 * 128;
    }
    __shared__ long long red[2][32];
    m = warp_sum(m);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = m;
        red[1][wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        m = lane < nw ? red[0][lane] : 0;
        b = lane < nw ? red[1][lane] : 0;
        m = warp_sum(m);
        b = warp_sum(b);
        if (lane == 0) {
            const int64_t RL = rec_len(g.L);
            atomicAdd(reinterpret_cast<unsigned long long *>(rec + r * RL + 1), (unsigned long long)m);
            atomicAdd(reinterpret_cast<unsigned long long *>(rec + r * RL + 2), (unsigned long long)b);
        }
    }
}

// ---------------------------------------------------------------------------------
// Axis correlation.  blockIdx.z = axis (0 = x, 1 = y, 2 = z), blockIdx.y = replica,
// blockIdx.x strides over panels of NC columns (a persistent grid).
//
// A column of L words is staged in shared memory extended to LE = L + NLB*RT words
// (element j holds col[j mod L]), at padded positions pad(j) = j + j/8 so that the
// stride-RT window loads below are bank-conflict free.  A work item is (column, block of
// RT consecutive lags r0..r0+RT-1): the item keeps a register window of the RT partner
// words col[j + r0 .. j + r0 + RT - 1] and slides it along j, so each step costs one
// broadcast load (col[j]) and one window load for RT XOR pairs.  The XOR words of each
// lag are summed either by POPC per word or by carry-save adders (Harley & Seal's
// popcount accumulation, one POPC per eight words); warps are split between the two so
// that the bit-count unit and the ALU are busy together.
__host__ __device__ inline int corr_nc(int L)
{
    int nc = 8192 / L;
    if (nc < 1) nc = 1;
    if (nc > 64) nc = 64;
    return nc;
}

__host__ __device__ inline int corr_rt(int L) { return L >= 8 ? 8 : 4; }
__host__ __device__ inline int corr_nlb(int L) { return (L / 2 + corr_rt(L) - 1) / corr_rt(L); }
__host__ __device__ inline int corr_le(int L) { return L + corr_nlb(L) * corr_rt(L); }
__host__ __device__ inline int corr_pad(int j) { return j + (j >> 3); }
__host__ __device__ inline int corr_lp(int L) { return corr_pad(corr_le(L) - 1) + 1; }

__host__ __device__ inline int64_t corr_ncols(const Geom &g, int axis)
{
    if (axis == 0) return ((int64_t)g.L * g.L + 31) / 32;  // 32-row bundles
    return 2 * (int64_t)g.L * g.W;                          // (pi, other coordinate, kw)
}

// Stage columns c0 .. c0+NC-1 of the y or z axis (column (pi, a, kw): a is z for the y
// axis, y for the z axis; element j is the other coordinate).  Consecutive threads take
// consecutive columns of one j, which are consecutive words in memory.
__device__ __forceinline__ void load_panel_yz(const uint32_t *S0, const uint32_t *S1, const Geom &g, int axis,
                                              int64_t c0, int NC, int64_t ncols, uint32_t *sm, int LE, int LP,
                                              int tid0, int stride)
{
    const int L = g.L, W = g.W;
    for (int e = tid0; e < NC * LE; e += stride) {
        const int j = e / NC;
        const int c = e - j * NC;
        const int64_t col = c0 + c;
        uint32_t v = 0u;
        if (col < ncols) {
            const int pi = (int)(col / ((int64_t)L * W));
            const int64_t rem = col - (int64_t)pi * L * W;
            const int a = (int)(rem / W);
            const int kw = (int)(rem - (int64_t)a * W);
            int jj = j;
            while (jj >= L) jj -= L;
            const int y = axis == 1 ? jj : a;
            const int z = axis == 1 ? a : jj;
            const uint32_t *Sq = ((pi + y + z) & 1) ? S1 : S0;
            v = __ldg(Sq + ((int64_t)z * L + y) * W + kw);
        }
        sm[c * LP + corr_pad(j)] = v;
    }
}

// Three CTAs per SM (80 registers): with that bound the compiler keeps the carry-save
// registers without spilling; two CTAs with more registers measured 3% slower.
// t + p * one with `one` = 1 passed at run time: the compiler cannot fold the product, so the
// sum issues as an integer multiply-add on the FMA pipe, which this kernel otherwise leaves
// idle, instead of an add on the integer ALU pipe that the XORs and adders saturate.
__device__ __forceinline__ uint32_t mad_u32(uint32_t p, uint32_t one, uint32_t t)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(p), "r"(one), "r"(t));
    return r;
}

template <int NT, int RT>
__global__ void __launch_bounds__(NT, 3) k_corr(const uint32_t *lat, Geom g, int64_t *rec, uint32_t one)
{
    extern __shared__ uint32_t csm[];
    const int axis = blockIdx.z;
    const int r = blockIdx.y;
    const int L = g.L, H = L / 2;
    const int NLB = corr_nlb(L), LE = corr_le(L), LP = corr_lp(L);
    const int NC = corr_nc(L);
    const uint32_t *S0 = lat + (2 * (int64_t)r) * g.nw;
    const uint32_t *S1 = S0 + g.nw;
    uint32_t *cols = csm;  // NC * LP words
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(csm + ((NC * LP + 1) & ~1));  // NLB*RT+1
    const int tid = threadIdx.x;
    for (int i = tid; i <= NLB * RT; i += NT) acc[i] = 0ull;
    const int64_t ncols = corr_ncols(g, axis);
    const int64_t npanels = (ncols + NC - 1) / NC;
    const int lane = tid & 31, wid = tid >> 5;
    for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
        __syncthreads();  // previous panel fully consumed
        const int64_t c0 = pnl * NC;
        const int nc = (int)min((int64_t)NC, ncols - c0);
        if (axis != 0) {
            load_panel_yz(S0, S1, g, axis, c0, NC, ncols, cols, LE, LP, tid, NT);
        } else {
            // bundle = rows 32b .. 32b+31 (row = y + L z); T[x] lane i = site (x, row 32b+i).
            // Tasks: (bundle, pi, kw), one warp each, 32 ballots per task.
            const int ntask = NC * 2 * g.W;
            for (int task = wid; task < ntask; task += NT / 32) {
                const int c = task / (2 * g.W);
                const int rem = task - c * 2 * g.W;
                const int pi = rem / g.W, kw = rem - pi * g.W;
                const int64_t row = (c0 + c) * 32 + lane;
                uint32_t v = 0u;
                if (c < nc && row < (int64_t)L * L) {
                    const int y = (int)(row % L), z = (int)(row / L);
                    const uint32_t *Sq = ((pi + y + z) & 1) ? S1 : S0;
                    v = __ldg(Sq + row * g.W + kw);
                }
                uint32_t mine = 0u;
                for (int k = 0; k < g.RB; ++k) {
                    const unsigned bal = __ballot_sync(0xffffffffu, (v >> k) & 1u);
                    if (lane == k) mine = bal;
                }
                if (lane < g.RB) {
                    const int x = 2 * (32 * kw + lane) + pi;
                    for (int j = x; j < LE; j += L) cols[c * LP + corr_pad(j)] = mine;
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < NC * NLB; e += NT) {
            const int c = e / NLB;
            const int r0 = 1 + (e - c * NLB) * RT;
            const uint32_t *col = cols + c * LP;
            uint32_t win[RT];
#pragma unroll
            for (int k = 0; k < RT; ++k) win[k] = col[corr_pad(r0 + k)];
            unsigned int total[RT];
            // Two ways to sum the XOR words, each saturating a different pipe: POPC per
            // word (bound by the 16-lane/clk bit-count unit) or carry-save adders (bound by
            // the ALU).  Warps 4..7 of every 8 take the carry-save path: warps w and w+4 share
            // an SM sub-partition, so each sub-partition runs one warp of each kind and both
            // pipes work at once; the choice is per warp, so no warp diverges.  (Measured at
            // L=2048: 4 of 8 on carry-save 148 ms, 3 of 8 166 ms, none 178 ms, per-item
            // alternation 7% slower than 3 of 8.)
            // Lags start at r0 = 1 + 8i, so the window's next word r0 + 7 + j + u sits at the
            // padded index 9(i + 1 + j/8) + u and the column word j + u at 9(j/8) + u: one
            // base pointer per 8-word step, the eight loads at immediate offsets.
            const uint32_t *wp = col + corr_pad(r0 + RT - 1);
            const uint32_t *ap = col;
            if (RT == 8 && (wid & 7) >= 4) {
                // Harley-Seal carry-save accumulation per lag: eight XOR words pass through
                // seven carry-save adders into (ones, twos, fours) and one "eights" word,
                // so one POPC covers eight words.
                uint32_t ones[RT], twos[RT], fours[RT], v[RT], twosA[RT], foursA[RT];
#pragma unroll
                for (int k = 0; k < RT; ++k) ones[k] = twos[k] = fours[k] = total[k] = 0u;
                for (int j = 0; j < L; j += RT, wp += 9, ap += 9) {
#pragma unroll
                    for (int u = 0; u < RT; ++u) {
                        if (u != 0 || j != 0) win[(u + RT - 1) % RT] = wp[u];
                        const uint32_t a = ap[u];
#pragma unroll
                        for (int k = 0; k < RT; ++k) {
                            const uint32_t x = a ^ win[(u + k) % RT];
                            if ((u & 1) == 0) {
                                v[k] = x;
                            } else {
                                // (carry, sum) of ones + v + x
                                const uint32_t t2 = (ones[k] & v[k]) | (x & (ones[k] ^ v[k]));
                                ones[k] = ones[k] ^ v[k] ^ x;
                                if (u == 1 || u == 5) {
                                    twosA[k] = t2;
                                } else {
                                    const uint32_t t4 = (twos[k] & twosA[k]) | (t2 & (twos[k] ^ twosA[k]));
                                    twos[k] = twos[k] ^ twosA[k] ^ t2;
                                    if (u == 3) {
                                        foursA[k] = t4;
                                    } else {
                                        const uint32_t t8 = (fours[k] & foursA[k]) | (t4 & (fours[k] ^ foursA[k]));
                                        fours[k] = fours[k] ^ foursA[k] ^ t4;
                                        total[k] = mad_u32(__popc(t8), one, total[k]);
                                    }
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < RT; ++k)
                    total[k] = 8u * total[k] + 4u * __popc(fours[k]) + 2u * __popc(twos[k]) + __popc(ones[k]);
            } else {
#pragma unroll
                for (int k = 0; k < RT; ++k) total[k] = 0u;
                if (RT == 8) {
                    for (int j = 0; j < L; j += RT, wp += 9, ap += 9) {
#pragma unroll
                        for (int u = 0; u < RT; ++u) {
                            if (u != 0 || j != 0) win[(u + RT - 1) % RT] = wp[u];
                            const uint32_t a = ap[u];
#pragma unroll
                            for (int k = 0; k < RT; ++k) total[k] = mad_u32(__popc(a ^ win[(u + k) % RT]), one, total[k]);
                        }
                    }
                } else {
                    for (int j = 0; j < L; j += RT) {
#pragma unroll
                        for (int u = 0; u < RT; ++u) {
                            const int jj = j + u;
                            if (u != 0 || j != 0) win[(u + RT - 1) % RT] = col[corr_pad(r0 + jj + RT - 1)];
                            const uint32_t a = col[corr_pad(jj)];
#pragma unroll
                            for (int k = 0; k < RT; ++k) total[k] += __popc(a ^ win[(u + k) % RT]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RT; ++k)
                if (total[k]) atomicAdd(acc + r0 + k, (unsigned long long)total[k]);
        }
    }
    __syncthreads();
    int64_t *D = rec + r * rec_len(L) + 3 + (int64_t)axis * (H + 1);
    for (int i = 1 + tid; i <= H; i += NT)
        if (acc[i]) atomicAdd(reinterpret_cast<unsigned long long *>(D + i), acc[i]);
}

static size_t corr_smem(int L)
{
    const int NC = corr_nc(L);
    const size_t words = ((size_t)NC * corr_lp(L) + 1) & ~(size_t)1;
    return words * 4 + (size_t)(corr_nlb(L) * corr_rt(L) + 1) * 8;
}

template <int RT>
static cudaError_t launch_corr(const uint32_t *lat, const Geom &g, int R, int64_t *rec, cudaStream_t s)
{
    const int L = g.L;
    const size_t smem = corr_smem(L);
    cudaError_t e = cudaFuncSetAttribute(k_corr<256, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_corr<256, RT>, 256, smem)) != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t maxc = corr_ncols(g, 0);
    if (corr_ncols(g, 1) > maxc) maxc = corr_ncols(g, 1);
    const int NC = corr_nc(L);
    int64_t panels = (maxc + NC - 1) / NC;
    // persistent: one resident wave over the 3 axes and R replicas
    int64_t want = ((int64_t)occ * sms) / ((int64_t)3 * R);
    if (want < 1) want = 1;
    if (panels > want) panels = want;
    k_corr<256, RT><<<dim3((unsigned)panels, (unsigned)R, 3), 256, smem, s>>>(lat, g, rec, 1u);
    return cudaGetLastError();
}

cudaError_t launch_measure(const uint32_t *lat, int L, int R, int64_t t, int corr, int64_t *rec, cudaStream_t s,
                           int64_t *launches, uint32_t *xt_scratch, int *err, double wait_timeout_s,
                           int inject_stall)
{
    const Geom g = make_geom(L);
    const int64_t RL = 3 + 3 * (int64_t)(L / 2 + 1);
    int64_t nb = (RL * R + 255) / 256;
    if (nb > 4096) nb = 4096;
    k_rec_init<<<(unsigned)nb, 256, 0, s>>>(rec, L, R, t, corr);
    if (L >= 256 && L % 256 == 0) {
        int64_t mb = (g.nw / 4 + 255) / 256;
        if (mb > (int64_t)device_sms() * 8) mb = (int64_t)device_sms() * 8;
        k_mb4<<<dim3((unsigned)mb, (unsigned)R), 256, 0, s>>>(lat, g, rec);
    } else {
        int64_t mb = (g.nw + 255) / 256;
        if (mb > (int64_t)device_sms() * 8) mb = (int64_t)device_sms() * 8;
        k_mb<<<dim3((unsigned)mb, (unsigned)R), 256, 0, s>>>(lat, g, rec);
    }
    int n = 2;
    if (corr == CORR_TENSOR) {
        if (!xt_scratch || !err || !corr_mma_supported(L)) return cudaErrorInvalidValue;
        const cudaError_t e = launch_corr_mma(lat, L, R, rec, xt_scratch, err, s, nullptr, wait_timeout_s, inject_stall);
        if (e != cudaSuccess) return e;
        n += 2;
    } else if (corr) {
        const cudaError_t e = corr_rt(L) == 8 ? launch_corr<8>(lat, g, R, rec, s) : launch_corr<4>(lat, g, R, rec, s);
        if (e != cudaSuccess) return e;
        ++n;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Derived quantities (double precision): e = -3 + 2B/N, m = M/N, l_E = N/B, and the
// first linear-interpolated crossing l_C of C(r) = sum_a (N - 2 D_a(r)) / (3N) (- m^2
// when connected) with the constant c (Results: c = 0.5).
__global__ void k_derived(const int64_t *rec, int L, int R, double c, bool connected, double *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t H = L / 2;
    const int64_t *q = rec + (int64_t)r * (3 + 3 * (H + 1));
    const double N = (double)L * (double)L * (double)L;
    const int64_t M = q[1], B = q[2];
    const int64_t *Dx = q + 3, *Dy = q + 3 + (H + 1), *Dz = q + 3 + 2 * (H + 1);
    const double m = __ddiv_rn((double)M, N);
    double *o = out + 4 * (int64_t)r;
    o[0] = __dadd_rn(-3.0, __ddiv_rn(__dmul_rn(2.0, (double)B), N));
    o[1] = m;
    o[2] = B == 0 ? __longlong_as_double(0x7ff0000000000000ll) : __ddiv_rn(N, (double)B);
    double lc = __longlong_as_double(0x7ff8000000000000ll);
    const double sub = connected ? __dmul_rn(m, m) : 0.0;
    const double N3 = __dmul_rn(3.0, N);
    if (Dx[0] >= 0) {
        for (int64_t k = 0; k < H; ++k) {
            const double g0 = __dadd_rn(__dadd_rn(__dsub_rn(N, __dmul_rn(2.0, (double)Dx[k])),
                                                  __dsub_rn(N, __dmul_rn(2.0, (double)Dy[k]))),
                                        __dsub_rn(N, __dmul_rn(2.0, (double)Dz[k])));
            const double g1 = __dadd_rn(__dadd_rn(__dsub_rn(N, __dmul_rn(2.0, (double)Dx[k + 1])),
                                                  __dsub_rn(N, __dmul_rn(2.0, (double)Dy[k + 1]))),
                                        __dsub_rn(N, __dmul_rn(2.0, (double)Dz[k + 1])));
            const double c0 = __dsub_rn(__ddiv_rn(g0, N3), sub);
            const double c1 = __dsub_rn(__ddiv_rn(g1, N3), sub);
            if (c0 >= c && c > c1) {
                lc = __dadd_rn((double)k, __ddiv_rn(__dsub_rn(c0, c), __dsub_rn(c0, c1)));
                break;
            }
        }
    }
    o[3] = lc;
}

cudaError_t launch_derived(const int64_t *rec, int L, int R, double c, bool connected, double *derived,
                           cudaStream_t s, int64_t *launches)
{
    k_derived<<<(R + 127) / 128, 128, 0, s>>>(rec, L, R, c, connected, derived);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace ising
