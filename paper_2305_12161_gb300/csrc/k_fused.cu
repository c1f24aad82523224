// One whole Monte Carlo sweep (both half-sweeps, Methods "Checkerboard update") in one pass
// over the lattice: temporal blocking of the red-black order.  The pass reads the store of
// sweep t (`cur`) and writes the store of sweep t+1 (`nxt`), so no CTA ever reads a value
// that another CTA of the same launch has already replaced.
//
// A CTA owns a tile of full rows and TZ planes (a z-block: the blocks of a launch hold
// L / nzb planes each, rounded per block) and marches along z.  With A the sublattice
// updated first and B the other, step k updates A on plane zA = z0 - 1 + k for the tile's
// rows and one halo row on each side, then B on plane zB = zA - 1 for the tile's rows; B's
// neighbours are A's new values of planes zB - 1 .. zB + 1, which this CTA has just
// computed, halo rows included.  A on the halo planes z0 - 1 and z0 + TZ and on the halo rows
// is computed but not stored: the CTA that owns them stores the same values.  Every update
// is the half-sweep's: same rule, same Philox bits (phase = the sublattice, counter word =
// the storage group), so the trajectory is bit-identical to two half-sweep launches.
//
// Per sweep the store is read once (plus L2-served halo rows and planes) and written once:
// N/4 bytes, against 3 N/8 for two half-sweeps.  The planes of the tile stream into shared
// memory by TMA bulk copies (cp.async.bulk, one per contiguous run of rows) issued by one
// thread and completing on mbarriers; every wait is bounded in wall time.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace ising {

namespace {

// x-neighbour words of the 128 sites of uint4 C: the same-k neighbour is C itself, the other
// is C shifted by one bit with the edge bit of the adjacent uint4 (direction by p).
__device__ __forceinline__ uint4 xshift(const uint4 &C, uint32_t edge_left_w, uint32_t edge_right_x, int p)
{
    uint4 X;
    if (p == 0) {
        X.x = __funnelshift_l(edge_left_w, C.x, 1);
        X.y = __funnelshift_l(C.x, C.y, 1);
        X.z = __funnelshift_l(C.y, C.z, 1);
        X.w = __funnelshift_l(C.z, C.w, 1);
    } else {
        X.x = __funnelshift_r(C.x, C.y, 1);
        X.y = __funnelshift_r(C.y, C.z, 1);
        X.z = __funnelshift_r(C.z, C.w, 1);
        X.w = __funnelshift_r(C.w, edge_right_x, 1);
    }
    return X;
}

// New spins of one uint4, as new_spins4 without the tie test: Glauber draws the group's
// Philox word from the launch's constant first rounds (the same word as philox4x32_10 of
// the counter (group, t, q, 0)).  The adders come before the draw, as in new_spins4: with
// the draw first the kernel ran 3% slower.
template <int RULE>
__device__ __forceinline__ uint4 fused_spins4(const uint4 &s, const uint4 &C, const uint4 &X, const uint4 &ym,
                                              const uint4 &yp, const uint4 &zm, const uint4 &zp, uint32_t group,
                                              const PhiloxLead &ld, const PhiloxKeys &keys)
{
    const uint32_t s1x = C.x ^ X.x ^ ym.x, c1x = maj3(C.x, X.x, ym.x);
    const uint32_t s1y = C.y ^ X.y ^ ym.y, c1y = maj3(C.y, X.y, ym.y);
    const uint32_t s1z = C.z ^ X.z ^ ym.z, c1z = maj3(C.z, X.z, ym.z);
    const uint32_t s1w = C.w ^ X.w ^ ym.w, c1w = maj3(C.w, X.w, ym.w);
    const uint32_t s2x = yp.x ^ zm.x ^ zp.x, c2x = maj3(yp.x, zm.x, zp.x);
    const uint32_t s2y = yp.y ^ zm.y ^ zp.y, c2y = maj3(yp.y, zm.y, zp.y);
    const uint32_t s2z = yp.z ^ zm.z ^ zp.z, c2z = maj3(yp.z, zm.z, zp.z);
    const uint32_t s2w = yp.w ^ zm.w ^ zp.w, c2w = maj3(yp.w, zm.w, zp.w);
    uint4 tau;
    if constexpr (RULE == TIE_GLAUBER) {
        const U4 o = philox4x32_10_lead(group, ld, keys);
        tau = make_uint4(s.x ^ o.x, s.y ^ o.y, s.z ^ o.z, s.w ^ o.w);
    } else if constexpr (RULE == TIE_ALWAYS) {
        tau = make_uint4(~s.x, ~s.y, ~s.z, ~s.w);
    } else {
        tau = s;
    }
    return make_uint4(maj3(c1x, c2x, maj3(s1x, s2x, tau.x)), maj3(c1y, c2y, maj3(s1y, s2y, tau.y)),
                      maj3(c1z, c2z, maj3(s1z, s2z, tau.z)), maj3(c1w, c2w, maj3(s1w, s2w, tau.w)));
}

}  // namespace

__device__ __forceinline__ uint64_t fused_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on phase `parity` of an mbarrier: spins on try_wait until the phase has
// completed or timeout_ns of %globaltimer have passed (with a cap on rounds as a backstop);
// false when it gave up.
__device__ __forceinline__ bool fused_mbar_wait(uint32_t addr, uint32_t parity, uint64_t timeout_ns)
{
    uint32_t done = 0;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(addr), "r"(parity)
                 : "memory");
    if (done) return true;
    const uint64_t t0 = fused_timer_ns();
    for (int it = 0; it < (1 << 28); ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63) == 63 && fused_timer_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// Bulk copy (TMA, non-tensor) of `bytes` from global to shared memory, completing on mbarrier
// `mbar`; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void fused_bulk(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// What differs between the replicas of a launch: kernel parameter space, so the Philox round
// keys are read as constant-bank operands of the round's logic operations and take no
// registers.
struct FusedRep {
    PhiloxKeys keys;           // round keys of the replica's Philox key (seed + replica)
    PhiloxLead leadA, leadB;   // the draws' constant first rounds for sweep t, phases A and B
    const uint4 *Acur, *Bcur;  // store of sweep t: first-updated sublattice A and the other, B
    uint4 *Anxt, *Bnxt;        // store of sweep t + 1
    uint32_t A;                // first sublattice (its tie-bit phase)
};

// Replicas one launch of the multi-replica form takes (grid.y); its parameters stay within
// the classic 4 KB parameter space.
constexpr int FUSED_MAXR = 16;

// Arguments of one launch: MR = 1, one replica; MR = FUSED_MAXR, replica blockIdx.y of rep.
template <int MR>
struct FusedArgs {
    FusedRep rep[MR];
    int L, nzb;                // z-blocks: block b holds planes b L / nzb .. (b + 1) L / nzb - 1
    uint32_t t;                // sweep index
    int *err;                  // set to 4 when a bounded wait gave up
    uint64_t timeout_ns;
};
static_assert(sizeof(FusedArgs<FUSED_MAXR>) <= 4096, "multi-replica parameters exceed 4 KB");

// Two tilings of the plane into row tiles.  First (BAL = false): a tile owns TY = 256 / W4
// rows y0 .. y0 + TY - 1, one per thread row, and lanes 0 .. 2 W4 - 1 of warp 0 also update A
// on the halo rows y0 - 1 and y0 + TY.  Balanced (BAL = true): the 256 / W4 thread rows are
// y0 - 1 .. y0 + 256 / W4 - 2, of which the outer two are the halo: every warp does the same
// work, the tile owns the TYB = 256 / W4 - 2 rows between them (the last tile owns the
// remainder of L and computes, without storing, rows past it).
template <int W4, bool BAL>
struct FusedTile {
    static constexpr int NR = 256 / W4;              // thread rows
    static constexpr int TYO = BAL ? NR - 2 : NR;    // rows a tile owns
    static constexpr int RA = BAL ? NR : NR + 2;     // A rows y0 - 1 .. : old A in a slot, new A
    static constexpr int RB = RA + 2;                // B rows y0 - 2 .. of a slot
    static constexpr int SLOT = (RB + RA) * W4;      // uint4 of a copy slot
};

// Shared memory: NS copy slots (a B plane and an old-A plane of the tile's rows), three
// slots of new A, NS mbarriers.
template <int W4, int NS, bool BAL>
static constexpr size_t fused_smem_bytes()
{
    using T = FusedTile<W4, BAL>;
    return sizeof(uint4) * (size_t)(NS * T::SLOT + 3 * T::RA * W4) + 8 * NS;
}

// Thread tid owns column cx = lane % W4 of one thread row (the rows of a warp share their
// parity, as in the half-sweep kernel) for both sublattices.  Copy group g (one TMA bulk copy
// per contiguous run of rows, issued by thread 0, completing on the mbarrier of slot g % NS)
// brings B plane z0 - 2 + g and, for g >= 2, old-A plane z0 - 1 + (g - 2); step k reads the
// slots of groups k, k + 1, k + 2 and, after the step's barrier, thread 0 refills the slot of
// group k - 1 with group k - 1 + NS, so NS - 3 groups stay in flight.  Every operand of a
// step comes from shared memory (nothing is carried across steps in registers), and the
// steps are unrolled in pairs so that the x direction P of the pair's two planes is a
// compile-time constant.  Offsets into a sublattice are 32-bit uint4 indices (L^3 / 256 < 2^31).
template <int RULE, int W4, int NS, int MINB, bool BAL, int MR>
__global__ void __launch_bounds__(256, MINB) k_mcs_fused(const __grid_constant__ FusedArgs<MR> fa)
{
    // first step whose wait gave up in some thread (0x7fffffff: none); every thread reads it
    // after the step's barrier and leaves when it is at or before its own step, so a failure
    // posted during step k + 1 by a thread that ran ahead is not seen as one of step k
    __shared__ int s_fail;
    using T = FusedTile<W4, BAL>;
    constexpr int RW = 32 / W4;
    constexpr int NR = T::NR, TYO = T::TYO, RA = T::RA, RB = T::RB, SLOT = T::SLOT;
    constexpr int NB = RB * W4;                // B items of a slot (A items follow)
    constexpr int NEW = RA * W4;               // items of a new-A slot
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr uint32_t HMASK = 2 * W4 >= 32 ? FULL : ((1u << (2 * W4)) - 1u);
    extern __shared__ __align__(16) uint4 fsm[];
    uint4 *ring = fsm;                   // [NS][SLOT], group g in slot g % NS
    uint4 *anew = fsm + NS * SLOT;       // [3][NEW], plane zA in slot k % 3
    uint64_t *full = reinterpret_cast<uint64_t *>(anew + 3 * NEW);  // [NS]
    pdl_enter();
    const FusedRep &rp = fa.rep[MR == 1 ? 0 : blockIdx.y];
    const int L = fa.L;
    const int tid = threadIdx.x;
    const int nty = (L + TYO - 1) / TYO;
    const int y0 = (int)(blockIdx.x % nty) * TYO;  // even: TYO is even
    const int nown = min(TYO, L - y0);
    const int zb = (int)(blockIdx.x / nty);
    const int z0 = (int)((int64_t)zb * L / fa.nzb);
    const int TZ = (int)((int64_t)(zb + 1) * L / fa.nzb) - z0;  // planes of this CTA's tile
    const int32_t plane4 = L * W4;
    const int32_t vol4 = L * plane4;
    auto wrapL = [&](int a) { return a < 0 ? a + L : (a >= L ? a - L : a); };
    const uint32_t full0 = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(ring);

    // thread 0: rows ystart .. ystart + n - 1 of the plane at `src` (wrapped in y) into dst, one
    // bulk copy per run of consecutive rows (up to three when the tile spans the whole plane)
    auto copy_rows = [&](uint32_t dst, const uint4 *src, int ystart, int n, uint32_t mbar) {
        int row = wrapL(ystart);
        while (n > 0) {
            const int m = min(n, L - row);
            fused_bulk(dst, src + row * W4, (uint32_t)(m * W4 * 16), mbar);
            dst += (uint32_t)(m * W4 * 16);
            n -= m;
            row = 0;
        }
    };
    int g_issued = -1;  // thread 0: last group issued
    auto issue = [&](int g) {  // thread 0
        if (g > TZ + 3) return;
        g_issued = g;
        const int sl = g % NS;
        const uint32_t mbar = full0 + 8u * (uint32_t)sl;
        const uint32_t bytes = (uint32_t)(16 * (NB + (g >= 2 ? RA * W4 : 0)));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
        const uint32_t dst = ring0 + (uint32_t)(16 * sl * SLOT);
        copy_rows(dst, rp.Bcur + wrapL(z0 - 2 + g) * plane4, y0 - 2, RB, mbar);
        if (g >= 2) copy_rows(dst + 16u * NB, rp.Acur + wrapL(z0 - 3 + g) * plane4, y0 - 1, RA, mbar);
    };
    if (tid == 0) {
        s_fail = 0x7fffffff;
        for (int i = 0; i < NS; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * (uint32_t)i));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int g = 0; g < NS; ++g) issue(g);

    const int warp = tid >> 5, lane = tid & 31;
    const int cx = lane & (W4 - 1);
    const int ty = (warp >> 1) * 2 * RW + (warp & 1) + 2 * (lane / W4);  // thread row
    const int yrow = BAL ? y0 - 1 + ty : y0 + ty;
    const int32_t own = wrapL(yrow) * W4 + cx;
    const int rN = (BAL ? ty : ty + 1) * W4 + cx;  // own row in an A slot
    const int rB = rN + W4;                        // own row in a B slot
    // new-A rows y - 1 and y + 1 of the B update (BAL: the halo rows have no outer neighbour;
    // their B is computed but not stored)
    const int rNm = (BAL && ty == 0) ? rN : rN - W4, rNp = (BAL && ty == NR - 1) ? rN : rN + W4;
    const bool bown = !BAL || (ty >= 1 && ty <= nown);  // B (and the stored A) of this row are the tile's
    const int srcl = (cx + W4 - 1) & (W4 - 1), srcr = (cx + 1) & (W4 - 1);
    // first tiling, halo lanes: row hr (0: y0-1, 1: y0+NR)
    const bool hl = !BAL && warp == 0 && lane < 2 * W4;
    const int hr = lane / W4;
    const int hB = (hr ? NR + 2 : 1) * W4 + cx;  // halo row in a B slot
    const int hN = (hr ? NR + 1 : 0) * W4 + cx;  // halo row in an A slot
    const int32_t dh = wrapL(hr ? y0 + NR : y0 - 1) * W4 + cx - own;
    const uint32_t A = rp.A;

    // groups 0 and 1 before the first step (step k waits for group k + 2); thread 0 tracks
    // the last group it saw land and the last it issued, for the drain after a failed wait
    bool bad = !fused_mbar_wait(full0, 0u, fa.timeout_ns);
    bad |= !fused_mbar_wait(full0 + 8u, 0u, fa.timeout_ns);
    int g_done = bad ? -1 : 1;
    int32_t oA = wrapL(z0 - 1) * plane4 + own;  // plane zA, own column
    // one step: A on plane zA = z0 - 1 + k (tile rows and halo rows), then B on zA - 1
    auto step = [&](const int k, auto Pc) -> bool {
        constexpr int P = decltype(Pc)::value;
        const int g2 = k + 2;
        // ring slots of groups k .. k + 2 and new-A slots of steps k, k - 1, k - 2, worked out
        // before the wait (measured 0.6% faster than where they are used)
        const int sl0 = k % NS, sl1 = (k + 1) % NS, sl2 = g2 % NS;
        const int na0 = k % 3, na1 = (k + 2) % 3, na2 = (k + 1) % 3;
        bool fail = !fused_mbar_wait(full0 + 8u * (uint32_t)sl2, (uint32_t)((g2 / NS) & 1), fa.timeout_ns);
        if (!fail) g_done = g2;
        // a plain barrier and a flag in shared memory: the barrier with an OR reduction
        // (__syncthreads_or) made the whole kernel 6% slower
        if (fail) atomicMin(&s_fail, k);
        __syncthreads();
        if (*(volatile int *)&s_fail <= k) return false;
        if (tid == 0 && k >= 1) issue(k - 1 + NS);  // the slot of group k - 1, last read in step k - 1
        const uint4 *S0 = ring + sl0 * SLOT;  // B plane zA - 1
        const uint4 *S1 = ring + sl1 * SLOT;  // B plane zA
        const uint4 *S2 = ring + sl2 * SLOT;  // B plane zA + 1; old A plane zA at NB
        uint4 *An = anew + na0 * NEW;
        const uint4 bm = S0[rB];
        uint4 a0;
        {
            const uint4 bc = S1[rB];
            const uint32_t e = __shfl_sync(FULL, P ? bc.x : bc.w, P ? srcr : srcl, W4);
            const uint4 X = xshift(bc, e, e, P);
            a0 = fused_spins4<RULE>(S2[NB + rN], bc, X, S1[rB - W4], S1[rB + W4], bm, S2[rB],
                                                (uint32_t)oA, rp.leadA, rp.keys);
            An[rN] = a0;
            if (bown && k >= 1 && k <= TZ) rp.Anxt[oA] = a0;
        }
        // first tiling, A on the halo rows: row y0 - 1 is odd (the other direction than warp
        // 0's even rows), row y0 + NR even (the same)
        if (hl) {
            const uint4 hbc = S1[hB];
            const int ph = P ^ 1 ^ hr;
            const uint32_t e = __shfl_sync(HMASK, ph ? hbc.x : hbc.w, ph ? srcr : srcl, W4);
            const uint4 X = xshift(hbc, e, e, ph);
            An[hN] = fused_spins4<RULE>(S2[NB + hN], hbc, X, S1[hB - W4], S1[hB + W4], S0[hB], S2[hB],
                                                    (uint32_t)(oA + dh), rp.leadA, rp.keys);
        }
        // B on plane zB = zA - 1, own column: new A of planes zB - 1, zB, zB + 1 are in the
        // new-A slots of steps k - 2 and k - 1, and a0
        if (k >= 2) {
            const uint4 *A1 = anew + na1 * NEW;  // step k - 1: plane zB
            const uint4 *A2 = anew + na2 * NEW;  // step k - 2: plane zB - 1
            const uint4 a1 = A1[rN];
            const uint32_t e = __shfl_sync(FULL, P ? a1.x : a1.w, P ? srcr : srcl, W4);
            const uint4 X = xshift(a1, e, e, P);
            const int32_t oB = oA >= plane4 ? oA - plane4 : oA - plane4 + vol4;
            const uint4 nb = fused_spins4<RULE>(bm, a1, X, A1[rNm], A1[rNp], A2[rN], a0, (uint32_t)oB, rp.leadB,
                                                rp.keys);
            if (bown) rp.Bnxt[oB] = nb;
        }
        oA += plane4;
        if (oA >= vol4) oA -= vol4;
        return true;
    };
    // x direction of A on plane zA at k = 0 (and of B on zA - 1): parity of yrow + zA + A,
    // yrow's parity is the warp's (plus one in the balanced tiling); it alternates with k
    const int p0 = ((warp & 1) + (BAL ? 1 : 0) + z0 - 1 + (int)A) & 1;
    bool ok = !__syncthreads_or(bad);
    if (ok) {
        // TZ + 2 steps in pairs; for odd TZ the last pair has one step
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        const int last = TZ + 1;
        if (p0) {
#pragma unroll 1
            for (int k = 0; k <= last && ok; k += 2) ok = step(k, I1{}) && (k + 1 > last || step(k + 1, I0{}));
        } else {
#pragma unroll 1
            for (int k = 0; k <= last && ok; k += 2) ok = step(k, I0{}) && (k + 1 > last || step(k + 1, I1{}));
        }
    }
    if (!ok && tid == 0) {
        // a wait gave up: report it, and let every bulk copy this CTA issued and did not see
        // land (groups g_done + 1 .. g_issued, at most NS of them, distinct slots) land,
        // bounded, before the CTA's shared memory is released
        atomicExch(fa.err, 4);
        for (int g = g_done + 1; g <= g_issued; ++g)
            fused_mbar_wait(full0 + 8u * (uint32_t)(g % NS), (uint32_t)((g / NS) & 1), fa.timeout_ns);
    }
}

// depth: copy groups in flight, 1..3 (0 = 2), plus 8 for the balanced tiling, plus 16 for
// z-blocks fitted to the resident CTAs (see fitted_zblocks).
bool fused_config_valid(int L, int TZ, int depth)
{
    return L >= 256 && L <= 2048 && L % 256 == 0 && (L & (L - 1)) == 0 && TZ >= 1 && L % TZ == 0 &&
           (depth & ~27) == 0;
}

// Number of z-blocks near L / TZ (within 25%) whose tile count nty * nzb fills the last wave
// of `slots` resident CTAs best (ties: the one nearest L / TZ).  Blocks then hold L / nzb
// planes, rounded per block: tiles of one launch differ by at most one plane, and the
// launch's last wave is nearly full instead of leaving SMs idle.
static int fitted_zblocks(int L, int TZ, int nty, int slots)
{
    const int nom = L / TZ;
    int best = nom;
    double best_eff = -1.0;
    for (int c = std::max(1, (3 * nom) / 4); c <= std::min(L / 2, (5 * nom + 3) / 4); ++c) {
        const int64_t ctas = (int64_t)nty * c;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff > best_eff + 1e-9 || (eff > best_eff - 1e-9 && std::abs(c - nom) < std::abs(best - nom))) {
            best_eff = eff;
            best = c;
        }
    }
    return best;
}

// Round keys of Philox key S on the host (the key words plus i Weyl increments).
static PhiloxKeys host_round_keys(uint64_t S)
{
    PhiloxKeys k;
    uint32_t a = (uint32_t)S, b = (uint32_t)(S >> 32);
    for (int i = 0; i < 10; ++i) {
        k.k0[i] = a;
        k.k1[i] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

// Kernel attributes of one instantiation, set once per process (the first call of a form).
template <class K>
static cudaError_t fused_attrs(K kern, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

static FusedRep fused_rep(const uint32_t *cur, uint32_t *nxt, int64_t nw, int r, uint64_t seed, int mixed,
                          uint32_t t)
{
    const uint64_t S = seed + (uint64_t)r;
    FusedRep a;
    a.keys = host_round_keys(S);
    a.A = mixed ? (uint32_t)mixed_first(S, t) : 0u;
    a.leadA = philox_lead(t, a.A, a.keys);
    a.leadB = philox_lead(t, 1u - a.A, a.keys);
    a.Acur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + a.A) * nw);
    a.Bcur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + 1 - a.A) * nw);
    a.Anxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + a.A) * nw);
    a.Bnxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + 1 - a.A) * nw);
    return a;
}

// One sweep of R replicas.  MULTI: up to FUSED_MAXR replicas per launch along grid.y, each
// with its own round keys, first sublattice and stores in the parameter array (for many
// small lattices, whose single-replica grids would leave most SMs idle); otherwise one launch
// per replica with its arguments as the kernel's only parameters.
template <int RULE, int W4, int NS, bool BAL, bool MULTI>
static cudaError_t fused_rule(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed, uint32_t t,
                              int TZ, bool fit, int *err, uint64_t timeout_ns, cudaStream_t s, bool pdl)
{
    constexpr int MR = MULTI ? FUSED_MAXR : 1;
    constexpr size_t smem = fused_smem_bytes<W4, NS, BAL>();
    // CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per CTA); the
    // registers are capped to match
    constexpr int MINB = (int)(233472 / (smem + 1024)) >= 4 ? 4 : 3;
    auto kern = k_mcs_fused<RULE, W4, NS, MINB, BAL, MR>;
    cudaError_t e = fused_attrs(kern, smem);
    if (e != cudaSuccess) return e;
    const Geom g = make_geom(L);
    constexpr int TYO = FusedTile<W4, BAL>::TYO;
    const int nty = (L + TYO - 1) / TYO;
    const int per_launch = MULTI ? std::min(R, FUSED_MAXR) : 1;
    int nzb = L / TZ;
    if (fit) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (e != cudaSuccess) return e;
        nzb = fitted_zblocks(L, TZ, nty * per_launch, std::max(1, per_sm) * device_sms());
    }
    for (int r0 = 0; r0 < R; r0 += per_launch) {
        const int nr = std::min(per_launch, R - r0);
        FusedArgs<MR> a;
        for (int i = 0; i < nr; ++i) a.rep[i] = fused_rep(cur, nxt, g.nw, r0 + i, seed, mixed, t);
        a.L = L;
        a.nzb = nzb;
        a.t = t;
        a.err = err;
        a.timeout_ns = timeout_ns;
        // programmatic dependent launch: the next sweep's CTAs are scheduled while this one
        // drains and wait in pdl_enter for its completion
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(nty * nzb), (unsigned)nr);
        lc.blockDim = dim3(256);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute attr[1] = {pdl_attribute()};
        lc.attrs = attr;
        lc.numAttrs = pdl ? 1 : 0;
        e = cudaLaunchKernelEx(&lc, kern, a);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <int RULE, int NS, bool BAL, bool MULTI>
static cudaError_t fused_one(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed, uint32_t t,
                             int TZ, bool fit, int *err, uint64_t timeout_ns, cudaStream_t s, bool pdl)
{
    switch (L / 256) {
    case 1: return fused_rule<RULE, 1, NS, BAL, MULTI>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 2: return fused_rule<RULE, 2, NS, BAL, MULTI>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 4: return fused_rule<RULE, 4, NS, BAL, MULTI>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 8: return fused_rule<RULE, 8, NS, BAL, MULTI>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    default: return cudaErrorInvalidValue;
    }
}

// Five-slot forms: several replicas per launch when there are several (the multi-replica
// kernel is built for these forms only).
template <int RULE, bool BAL>
static cudaError_t fused_five(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed, uint32_t t,
                              int TZ, bool fit, int *err, uint64_t timeout_ns, cudaStream_t s, bool pdl)
{
    if (R > 1) return fused_one<RULE, 5, BAL, true>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    return fused_one<RULE, 5, BAL, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
}

// depth = copy groups in flight while a step computes: 1..3 (four to six slots; 0 = 2); +8:
// the balanced tiling; +16: z-blocks fitted to the resident CTAs
template <int RULE>
static cudaError_t fused_depth(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed,
                               uint32_t t, int TZ, int depth, int *err, uint64_t timeout_ns, cudaStream_t s, bool pdl)
{
    const bool fit = depth & 16;
    switch (depth & ~16) {
    case 1: return fused_one<RULE, 4, false, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 3: return fused_one<RULE, 6, false, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 9: return fused_one<RULE, 4, true, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 8:
    case 10: return fused_five<RULE, true>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    case 11: return fused_one<RULE, 6, true, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    default: return fused_five<RULE, false>(cur, nxt, L, R, seed, mixed, t, TZ, fit, err, timeout_ns, s, pdl);
    }
}

// Launches of one sweep of R replicas: the five-slot forms take up to FUSED_MAXR replicas per
// launch, the others one.
static int64_t fused_launches_per_sweep(int R, int depth)
{
    const int d = depth & ~16;
    const bool five = !(d == 1 || d == 3 || d == 9 || d == 11);
    return five && R > 1 ? (R + FUSED_MAXR - 1) / FUSED_MAXR : R;
}

cudaError_t launch_sweeps_fused(uint32_t **cur, uint32_t **nxt, int L, int R, uint64_t seed, int rule, int64_t t0,
                                int64_t n_mcs, int cycle, int TZ, int depth, int *err, double timeout_s,
                                cudaStream_t s, int64_t *launches, bool pdl)
{
    const uint64_t timeout_ns = (uint64_t)(timeout_s * 1e9);
    for (int64_t k = 0; k < n_mcs; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        cudaError_t e;
        switch (rule) {
        case TIE_GLAUBER:
            e = fused_depth<TIE_GLAUBER>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, err, timeout_ns, s, pdl);
            break;
        case TIE_ALWAYS:
            e = fused_depth<TIE_ALWAYS>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, err, timeout_ns, s, pdl);
            break;
        default: e = fused_depth<TIE_NEVER>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, err, timeout_ns, s, pdl); break;
        }
        if (e != cudaSuccess) return e;
        uint32_t *tmp = *cur;  // the new sweep becomes the current store
        *cur = *nxt;
        *nxt = tmp;
        if (launches) *launches += fused_launches_per_sweep(R, depth);
    }
    return cudaSuccess;
}

}  // namespace ising
