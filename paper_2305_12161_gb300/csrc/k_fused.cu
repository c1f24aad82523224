// One whole Monte Carlo sweep (both half-sweeps, Methods "Checkerboard update") in one pass
// over the lattice: temporal blocking of the red-black order.  The pass reads the store of
// sweep t (`cur`) and writes the store of sweep t+1 (`nxt`), so no CTA ever reads a value
// that another CTA of the same launch has already replaced.
//
// A CTA owns TY full rows and TZ planes and marches along z.  With A the sublattice updated
// first and B the other, step k updates A on plane zA = z0 - 1 + k for the tile's rows and
// one halo row on each side, then B on plane zB = zA - 1 for the tile's rows; B's neighbours
// are A's new values of planes zB - 1 .. zB + 1, which this CTA has just computed, halo
// rows included.  A on the halo planes z0 - 1 and z0 + TZ and on the halo rows is computed
// but not stored: the CTA that owns them stores the same values.  Every update is the
// half-sweep's: same rule, same Philox bits (phase = the sublattice, counter word = the
// storage group), so the trajectory is bit-identical to two half-sweep launches.
//
// Per sweep the store is read once (plus L2-served halo rows and planes) and written once:
// N/4 bytes, against 3 N/8 for two half-sweeps.  Two tilings: k_mcs_fused (tiles of
// 256 / W4 rows, the halo rows of A on extra lanes of warp 0) and k_mcs_fused_bal (256 / W4
// computed rows of which the outer two are the halo, so every warp does the same work).
#include "common.cuh"
#include "kernels.h"

namespace ising {

namespace {

__device__ __forceinline__ void fcp16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void fcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void fwait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

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

}  // namespace

// Shared memory: NS copy slots, each one B plane (rows y0-2 .. y0+TY+1) and one old-A plane
// (rows y0-1 .. y0+TY); two slots of new A (rows y0-1 .. y0+TY).
template <int W4, int NS>
static constexpr size_t fused_smem_bytes()
{
    constexpr int TY = 256 / W4;
    return sizeof(uint4) * (size_t)(NS * (2 * TY + 6) * W4 + 2 * (TY + 2) * W4);
}

// Thread tid owns column cx = lane % W4 of row y0 + ty (the rows of a warp share their parity,
// as in the half-sweep kernel) for both sublattices, so the B update finds its own column's
// new A on planes zB - 1, zB, zB + 1 in registers and reads only rows y +- 1 from shared memory.
// x-edge words come from the neighbouring lane of the row by a shuffle.  Lanes 0 .. 2 W4 - 1
// of warp 0 also update A on the halo rows.  Copy group g brings B plane z0 - 2 + g and, for
// g >= 2, old-A plane z0 - 1 + (g - 2); step k reads the slots of groups k .. k + 2 and
// refills the slot of group k - 1 with group k + NS - 1, so NS - 3 groups stay in flight.
// Offsets into a sublattice are 32-bit uint4 indices (L^3 / 256 < 2^31).
template <int RULE, int W4, int NS>
__global__ void __launch_bounds__(256, 3) k_mcs_fused(const uint32_t *__restrict__ cur, uint32_t *__restrict__ nxt,
                                                      Geom g, int mixed, uint32_t t, uint64_t seed, int TZ)
{
    constexpr int NT = 256, TY = NT / W4, RW = 32 / W4;
    constexpr int RB = TY + 4;                 // B rows of a slot
    constexpr int RA = TY + 2;                 // A rows of a slot, and of a new-A slot
    constexpr int NB = RB * W4;                // B items of a slot (A items follow)
    constexpr int SLOT = (RB + RA) * W4;
    constexpr int NCP = (SLOT + NT - 1) / NT;  // copies per thread per group
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr uint32_t HMASK = 2 * W4 >= 32 ? FULL : ((1u << (2 * W4)) - 1u);
    extern __shared__ uint4 fsm[];
    uint4 *ring = fsm;              // [NS][SLOT], group g in slot g % NS
    uint4 *anew = fsm + NS * SLOT;  // [2][RA * W4]
    const int L = g.L;
    const int tid = threadIdx.x;
    const int nty = L / TY;
    const int y0 = (int)(blockIdx.x % nty) * TY;
    const int z0 = (int)(blockIdx.x / nty) * TZ;
    const int r = blockIdx.y;
    const uint64_t S = seed + (uint64_t)r;
    // sublattice updated first: 0 (01 cycle) or the sweep's drawn order (mixed cycle)
    int A = 0;
    if (mixed) A = (int)(philox4x32_10(0u, t, 5u, 0u, (uint32_t)S, (uint32_t)(S >> 32)).x & 1u);
    const int B = 1 - A;
    const int32_t plane4 = L * W4;
    const int32_t vol4 = L * plane4;
    const uint4 *Acur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + A) * g.nw);
    const uint4 *Bcur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + B) * g.nw);
    uint4 *Anxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + A) * g.nw);
    uint4 *Bnxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + B) * g.nw);
    const PhiloxKeys keys = philox_keys(S);
    auto wrapL = [&](int a) { return a < 0 ? a + L : (a >= L ? a - L : a); };

    // copies: slot item e = tid + j NT; its offset within a plane is fixed over the march
    int32_t coff[NCP];
#pragma unroll
    for (int j = 0; j < NCP; ++j) {
        const int e = tid + j * NT;
        const int ea = e < NB ? e : e - NB;
        coff[j] = wrapL(y0 + ea / W4 - (e < NB ? 2 : 1)) * W4 + (ea & (W4 - 1));
    }
    int32_t ob = wrapL(z0 - 2) * plane4;  // B plane of the next group
    int32_t oa = wrapL(z0 - 1) * plane4;  // A plane of the next group that has one
    auto issue = [&](int gi, int slot) {
        uint4 *dst = ring + slot * SLOT;
        if (gi <= TZ + 3) {
            const bool wa = gi >= 2;
#pragma unroll
            for (int j = 0; j < NCP; ++j) {
                const int e = tid + j * NT;
                if (e < NB)
                    fcp16(dst + e, Bcur + (ob + coff[j]));
                else if (e < SLOT && wa)
                    fcp16(dst + e, Acur + (oa + coff[j]));
            }
            ob += plane4;
            if (ob == vol4) ob = 0;
            if (wa) {
                oa += plane4;
                if (oa == vol4) oa = 0;
            }
        }
        fcommit();
    };

    const int warp = tid >> 5, lane = tid & 31;
    const int cx = lane & (W4 - 1);
    const int ty = (warp >> 1) * 2 * RW + (warp & 1) + 2 * (lane / W4);
    const int32_t own = (y0 + ty) * W4 + cx;
    const int rB = (ty + 2) * W4 + cx;  // own row in a B slot
    const int rN = (ty + 1) * W4 + cx;  // own row in an A slot
    const int srcl = (cx + W4 - 1) & (W4 - 1), srcr = (cx + 1) & (W4 - 1);
    // halo lanes: row hr (0: y0-1, 1: y0+TY)
    const bool hl = warp == 0 && lane < 2 * W4;
    const int hr = lane / W4;
    const int hB = (hr ? TY + 2 : 1) * W4 + cx;  // halo row in a B slot
    const int hN = (hr ? TY + 1 : 0) * W4 + cx;  // halo row in an A slot
    const int32_t dh = wrapL(hr ? y0 + TY : y0 - 1) * W4 + cx - own;

#pragma unroll 1
    for (int gi = 0; gi < NS - 1; ++gi) issue(gi, gi);
    int32_t oA = wrapL(z0 - 1) * plane4 + own;  // plane zA, own column
    int32_t oB = 0;                             // plane zA - 1 (= zB), own column
    int p = (ty + z0 - 1 + A) & 1;              // x direction on plane zA (y0 even); also B's on zA - 1
    fwait<NS - 3>();  // groups 0 and 1
    __syncthreads();
    uint4 bm = ring[0 * SLOT + rB];  // B plane zA - 1, own column
    uint4 bc = ring[1 * SLOT + rB];  // B plane zA
    uint4 a1 = make_uint4(0u, 0u, 0u, 0u), a2 = a1;  // new A, planes zA - 1 and zA - 2, own column
    int sl0 = 0;  // slot of group k
#pragma unroll 1
    for (int k = 0; k <= TZ + 1; ++k) {
        fwait<NS - 4>();  // group k + 2 has landed
        __syncthreads();
        const int sl1 = sl0 == NS - 1 ? 0 : sl0 + 1, sl2 = sl1 == NS - 1 ? 0 : sl1 + 1;
        issue(k + NS - 1, sl0 == 0 ? NS - 1 : sl0 - 1);  // the slot of group k - 1, last read in step k - 1
        const uint4 *Bsm = ring + sl0 * SLOT;  // B plane zA - 1
        const uint4 *Bs0 = ring + sl1 * SLOT;  // B plane zA
        const uint4 *Bsp = ring + sl2 * SLOT;  // B plane zA + 1, old A plane zA (at NB)
        sl0 = sl1;
        uint4 *An = anew + (k & 1) * RA * W4;
        // A, own column
        const uint4 bp = Bsp[rB];
        uint4 a0;
        {
            const uint32_t e = __shfl_sync(FULL, p ? bc.x : bc.w, p ? srcr : srcl, W4);
            const uint4 X = xshift(bc, e, e, p);
            a0 = new_spins4<RULE, false>(Bsp[NB + rN], bc, X, Bs0[rB - W4], Bs0[rB + W4], bm, bp, (uint32_t)oA, t,
                               (uint32_t)A, keys);
            An[rN] = a0;
            if (k >= 1 && k <= TZ) Anxt[oA] = a0;
        }
        // A, halo rows: row y0 - 1 is odd (the other direction than warp 0's even rows), row
        // y0 + TY even (the same)
        if (hl) {
            const uint4 hbc = Bs0[hB];
            const int ph = p ^ 1 ^ hr;
            const uint32_t e = __shfl_sync(HMASK, ph ? hbc.x : hbc.w, ph ? srcr : srcl, W4);
            const uint4 X = xshift(hbc, e, e, ph);
            An[hN] = new_spins4<RULE, false>(Bsp[NB + hN], hbc, X, Bs0[hB - W4], Bs0[hB + W4], Bsm[hB], Bsp[hB],
                                   (uint32_t)(oA + dh), t, (uint32_t)A, keys);
        }
        // B on plane zB = zA - 1, own column: new A of planes zB - 1, zB, zB + 1 are a2, a1, a0
        if (k >= 2) {
            const uint4 *Ap = anew + ((k - 1) & 1) * RA * W4;  // new A, plane zB
            const uint32_t e = __shfl_sync(FULL, p ? a1.x : a1.w, p ? srcr : srcl, W4);
            const uint4 X = xshift(a1, e, e, p);
            Bnxt[oB] = new_spins4<RULE, false>(bm, a1, X, Ap[rN - W4], Ap[rN + W4], a2, a0, (uint32_t)oB, t, (uint32_t)B, keys);
        }
        a2 = a1;
        a1 = a0;
        bm = bc;
        bc = bp;
        oB = oA;
        oA += plane4;
        if (oA >= vol4) oA -= vol4;
        p ^= 1;
    }
    fwait<0>();
}

// Balanced tiling.  The CTA computes the first sublattice on NA = 256 / W4 rows,
// y0 - 1 .. y0 + NA - 2, and the second on the NA - 2 rows between them it owns, so the two
// halo rows are ordinary thread rows: every warp updates one A and one B column per step, and
// no warp waits at the barrier for another's extra work.  Tiles of NA - 2 rows do not divide
// L: the last tile owns the remainder and computes (but does not store) rows past it.
template <int W4, int NS>
static constexpr size_t fused_bal_smem_bytes()
{
    return sizeof(uint4) * (size_t)(NS * (512 + 2 * W4) + 2 * 256);
}

template <int RULE, int W4, int NS, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_mcs_fused_bal(const uint32_t *__restrict__ cur, uint32_t *__restrict__ nxt, Geom g, int mixed, uint32_t t,
                    uint64_t seed, int TZ)
{
    constexpr int NT = 256, NA = NT / W4, TYB = NA - 2, RW = 32 / W4;
    constexpr int RB = NA + 2;          // B rows of a slot: y0 - 2 .. y0 + NA - 1
    constexpr int NB = RB * W4;         // B items of a slot; NT old-A items follow (NA rows)
    constexpr int SLOT = NB + NT;       // = 512 + 2 W4
    constexpr int NX = SLOT - 2 * NT;   // items past two per thread, on the last NX threads
    constexpr uint32_t FULL = 0xffffffffu;
    extern __shared__ uint4 fsm[];
    uint4 *ring = fsm;              // [NS][SLOT], group g in slot g % NS
    uint4 *anew = fsm + NS * SLOT;  // [2][NT]: new A of the NA rows
    const int L = g.L;
    const int tid = threadIdx.x;
    const int nty = (L + TYB - 1) / TYB;
    const int y0 = (int)(blockIdx.x % nty) * TYB;  // even: TYB is even
    const int nown = min(TYB, L - y0);
    const int z0 = (int)(blockIdx.x / nty) * TZ;
    const int r = blockIdx.y;
    const uint64_t S = seed + (uint64_t)r;
    // sublattice updated first: 0 (01 cycle) or the sweep's drawn order (mixed cycle)
    int A = 0;
    if (mixed) A = (int)(philox4x32_10(0u, t, 5u, 0u, (uint32_t)S, (uint32_t)(S >> 32)).x & 1u);
    const int B = 1 - A;
    const int32_t plane4 = L * W4;
    const int32_t vol4 = L * plane4;
    const uint4 *Acur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + A) * g.nw);
    const uint4 *Bcur = reinterpret_cast<const uint4 *>(cur + (2 * (int64_t)r + B) * g.nw);
    uint4 *Anxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + A) * g.nw);
    uint4 *Bnxt = reinterpret_cast<uint4 *>(nxt + (2 * (int64_t)r + B) * g.nw);
    const PhiloxKeys keys = philox_keys(S);
    auto wrapL = [&](int a) { return a < 0 ? a + L : (a >= L ? a - L : a); };
    // slot item e -> its offset within a plane (fixed over the march)
    auto item_off = [&](int e) {
        return e < NB ? wrapL(y0 - 2 + e / W4) * W4 + (e & (W4 - 1))
                      : wrapL(y0 - 1 + (e - NB) / W4) * W4 + ((e - NB) & (W4 - 1));
    };
    const int32_t coff0 = item_off(tid), coff1 = item_off(tid + NT);
    const bool cx3 = tid >= NT - NX;
    const int e3 = 2 * NT + tid - (NT - NX);
    const int32_t coff3 = item_off(cx3 ? e3 : 0);
    int32_t ob = wrapL(z0 - 2) * plane4;  // B plane of the next group
    int32_t oa = wrapL(z0 - 1) * plane4;  // A plane of the next group that has one
    auto issue = [&](int gi, int slot) {
        uint4 *dst = ring + slot * SLOT;
        if (gi <= TZ + 3) {
            const bool wa = gi >= 2;
            fcp16(dst + tid, Bcur + (ob + coff0));  // tid < NB
            if (tid + NT < NB)
                fcp16(dst + tid + NT, Bcur + (ob + coff1));
            else if (wa)
                fcp16(dst + tid + NT, Acur + (oa + coff1));
            if (cx3 && wa) fcp16(dst + e3, Acur + (oa + coff3));
            ob += plane4;
            if (ob == vol4) ob = 0;
            if (wa) {
                oa += plane4;
                if (oa == vol4) oa = 0;
            }
        }
        fcommit();
    };

    const int warp = tid >> 5, lane = tid & 31;
    const int cx = lane & (W4 - 1);
    const int ty = (warp >> 1) * 2 * RW + (warp & 1) + 2 * (lane / W4);  // A row: y0 - 1 + ty
    const int32_t own = wrapL(y0 - 1 + ty) * W4 + cx;
    const bool bown = ty >= 1 && ty <= nown;  // B (and the stored A) of this row are the tile's
    const int rB = (ty + 1) * W4 + cx;        // the row in a B slot
    const int rA = NB + ty * W4 + cx;         // the row's old A in a slot
    const int rN = ty * W4 + cx;              // the row in a new-A slot
    const int rNm = ty >= 1 ? rN - W4 : rN, rNp = ty <= NA - 2 ? rN + W4 : rN;
    const int srcl = (cx + W4 - 1) & (W4 - 1), srcr = (cx + 1) & (W4 - 1);

#pragma unroll 1
    for (int gi = 0; gi < NS - 1; ++gi) issue(gi, gi);
    int32_t oz = wrapL(z0 - 1) * plane4;  // plane zA
    int32_t ozB = 0;                      // plane zA - 1 (= zB)
    int p = (ty + 1 + z0 - 1 + A) & 1;    // x direction of A on (y0 - 1 + ty, zA), and of B on zA - 1
    fwait<NS - 3>();  // groups 0 and 1
    __syncthreads();
    uint4 bm = ring[0 * SLOT + rB];  // B plane zA - 1, own column
    uint4 bc = ring[1 * SLOT + rB];  // B plane zA
    uint4 a1 = make_uint4(0u, 0u, 0u, 0u), a2 = a1;  // new A, planes zA - 1 and zA - 2, own column
    int sl0 = 0;  // slot of group k
#pragma unroll 1
    for (int k = 0; k <= TZ + 1; ++k) {
        fwait<NS - 4>();  // group k + 2 has landed
        __syncthreads();
        const int sl1 = sl0 == NS - 1 ? 0 : sl0 + 1, sl2 = sl1 == NS - 1 ? 0 : sl1 + 1;
        issue(k + NS - 1, sl0 == 0 ? NS - 1 : sl0 - 1);  // the slot of group k - 1, last read in step k - 1
        const uint4 *Bs0 = ring + sl1 * SLOT;  // B plane zA
        const uint4 *Bsp = ring + sl2 * SLOT;  // B plane zA + 1, old A plane zA
        sl0 = sl1;
        uint4 *An = anew + (k & 1) * NT;
        // A, own column
        const uint4 bp = Bsp[rB];
        const uint32_t e = __shfl_sync(FULL, p ? bc.x : bc.w, p ? srcr : srcl, W4);
        const uint4 X = xshift(bc, e, e, p);
        const uint4 a0 = new_spins4<RULE, false>(Bsp[rA], bc, X, Bs0[rB - W4], Bs0[rB + W4], bm, bp, (uint32_t)(oz + own), t,
                                       (uint32_t)A, keys);
        An[rN] = a0;
        if (bown && k >= 1 && k <= TZ) Anxt[oz + own] = a0;
        // B on plane zB = zA - 1, own column: new A of planes zB - 1, zB, zB + 1 are a2, a1, a0
        if (k >= 2) {
            const uint4 *Ap = anew + ((k - 1) & 1) * NT;  // new A, plane zB
            const uint32_t eb = __shfl_sync(FULL, p ? a1.x : a1.w, p ? srcr : srcl, W4);
            const uint4 Xb = xshift(a1, eb, eb, p);
            const uint4 nb = new_spins4<RULE, false>(bm, a1, Xb, Ap[rNm], Ap[rNp], a2, a0, (uint32_t)(ozB + own), t,
                                           (uint32_t)B, keys);
            if (bown) Bnxt[ozB + own] = nb;
        }
        a2 = a1;
        a1 = a0;
        bm = bc;
        bc = bp;
        ozB = oz;
        oz += plane4;
        if (oz == vol4) oz = 0;
        p ^= 1;
    }
    fwait<0>();
}

// depth: copy groups in flight (2 or 3; 0 = 2), plus 8 for the balanced tiling
bool fused_config_valid(int L, int TZ, int depth)
{
    const int d = depth & ~8;
    return L >= 256 && L <= 2048 && L % 256 == 0 && (L & (L - 1)) == 0 && TZ >= 1 && L % TZ == 0 &&
           (d == 0 || d == 2 || d == 3) && (depth & ~11) == 0;
}

template <int RULE, int W4, int NS>
static cudaError_t fused_bal_rule(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed,
                                  uint32_t t, int TZ, cudaStream_t s)
{
    constexpr size_t smem = fused_bal_smem_bytes<W4, NS>();
    // five slots fit four CTAs per SM: registers capped for them
    auto kern = k_mcs_fused_bal<RULE, W4, NS, NS == 5 ? 4 : 3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const Geom g = make_geom(L);
    constexpr int TYB = 256 / W4 - 2;
    const dim3 grid((unsigned)(((L + TYB - 1) / TYB) * (L / TZ)), (unsigned)R);
    kern<<<grid, 256, smem, s>>>(cur, nxt, g, mixed, t, seed, TZ);
    return cudaGetLastError();
}

template <int RULE, int W4, int NS>
static cudaError_t fused_rule(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed, uint32_t t,
                              int TZ, cudaStream_t s)
{
    constexpr size_t smem = fused_smem_bytes<W4, NS>();
    cudaError_t e =
        cudaFuncSetAttribute(k_mcs_fused<RULE, W4, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)  // shared memory for 3 CTAs per SM (the rest stays L1)
        e = cudaFuncSetAttribute(k_mcs_fused<RULE, W4, NS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const Geom g = make_geom(L);
    constexpr int TY = 256 / W4;
    const dim3 grid((unsigned)((L / TY) * (L / TZ)), (unsigned)R);
    k_mcs_fused<RULE, W4, NS><<<grid, 256, smem, s>>>(cur, nxt, g, mixed, t, seed, TZ);
    return cudaGetLastError();
}

template <int RULE, int NS, bool BAL>
static cudaError_t fused_one(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed, uint32_t t,
                             int TZ, cudaStream_t s)
{
    switch (L / 256) {
    case 1: return BAL ? fused_bal_rule<RULE, 1, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s)
                       : fused_rule<RULE, 1, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    case 2: return BAL ? fused_bal_rule<RULE, 2, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s)
                       : fused_rule<RULE, 2, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    case 4: return BAL ? fused_bal_rule<RULE, 4, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s)
                       : fused_rule<RULE, 4, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    case 8: return BAL ? fused_bal_rule<RULE, 8, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s)
                       : fused_rule<RULE, 8, NS>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    default: return cudaErrorInvalidValue;
    }
}

// depth = copy groups in flight while a step computes: 2 (five slots) or 3 (six); +8: the
// balanced tiling
template <int RULE>
static cudaError_t fused_depth(const uint32_t *cur, uint32_t *nxt, int L, int R, uint64_t seed, int mixed,
                               uint32_t t, int TZ, int depth, cudaStream_t s)
{
    switch (depth) {
    case 3: return fused_one<RULE, 6, false>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    case 8:
    case 10: return fused_one<RULE, 5, true>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    case 11: return fused_one<RULE, 6, true>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    default: return fused_one<RULE, 5, false>(cur, nxt, L, R, seed, mixed, t, TZ, s);
    }
}

cudaError_t launch_sweeps_fused(uint32_t **cur, uint32_t **nxt, int L, int R, uint64_t seed, int rule, int64_t t0,
                                int64_t n_mcs, int cycle, int TZ, int depth, cudaStream_t s, int64_t *launches)
{
    for (int64_t k = 0; k < n_mcs; ++k) {
        const uint32_t t = (uint32_t)(t0 + k);
        cudaError_t e;
        switch (rule) {
        case TIE_GLAUBER: e = fused_depth<TIE_GLAUBER>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, s); break;
        case TIE_ALWAYS: e = fused_depth<TIE_ALWAYS>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, s); break;
        default: e = fused_depth<TIE_NEVER>(*cur, *nxt, L, R, seed, cycle, t, TZ, depth, s); break;
        }
        if (e != cudaSuccess) return e;
        uint32_t *tmp = *cur;  // the new sweep becomes the current store
        *cur = *nxt;
        *nxt = tmp;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace ising
