// Device-side building blocks shared by the library's kernels: the lattice geometry of
// the 1-bit sublattice store, Philox4x32-10, the random word of a storage word, and
// the bit-sliced six-neighbour majority of the T -> 0 Glauber rule.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

// Streaming multiprocessors of the current device (looked up once per device), for grid
// caps and tile heuristics.  1 if the query fails: every kernel sized by it strides over
// its work, so a small grid is slower, never wrong.
inline int device_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

enum Rule : int { TIE_GLAUBER = 0, TIE_ALWAYS = 1, TIE_NEVER = 2 };

// Geometry of one lattice in the packed store.
//   Sublattice q = (x+y+z) mod 2 holds the N/2 sites x = 2k + p, p = (y+z+q) mod 2,
//   k = 0..L/2-1 of every row (y,z).  Row index row = y + L*z.
//   L >= 64 (multiple of 64): a row is W = L/64 words of 32 bits, bit b of word kw is
//   k = 32*kw + b, so storage word sw = row*W + kw is exactly compressed-index word
//   h >> 5 of the sites it holds.
//   L in {4,8,16,32}: a row is one word holding its RB = L/2 sites in bits 0..RB-1.
struct Geom {
    int L;
    int W;        // words per row
    int RB;       // valid bits per word (32, or L/2 for L < 64)
    int64_t nw;   // words per sublattice = L*L*W
};

__host__ __device__ inline Geom make_geom(int L)
{
    Geom g;
    g.L = L;
    g.W = L >= 64 ? L / 64 : 1;
    g.RB = L >= 64 ? 32 : L / 2;
    g.nw = (int64_t)L * L * g.W;
    return g;
}

__host__ __device__ inline uint32_t row_mask(int RB) { return RB >= 32 ? 0xffffffffu : ((1u << RB) - 1u); }

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64-bit
// products of counter words 0 and 2 with the round multipliers, the high halves mixed
// into words 1 and 3 with the round key; the key advances by the Weyl constants.
struct U4 {
    uint32_t x, y, z, w;
};

// High and low halves of the 32 x 32 -> 64-bit product.  On the device the two halves are
// asked for separately (a high multiply and a plain multiply): written as one 64-bit product
// the round issued 12% more instructions in the sweep kernels.
__host__ __device__ __forceinline__ void mul_hi_lo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    const uint64_t p = (uint64_t)a * b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                     uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t h0, l0, h1, l1;
        mul_hi_lo(M0, c0, h0, l0);
        mul_hi_lo(M1, c2, h1, l1);
        const uint32_t n0 = h1 ^ c1 ^ k0;
        const uint32_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += W0;
        k1 += W1;
    }
    return U4{c0, c1, c2, c3};
}

// The ten round keys of one Philox key, computed once and reused for many counters.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint64_t S)
{
    PhiloxKeys k;
    uint32_t a = (uint32_t)S, b = (uint32_t)(S >> 32);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        k.k0[i] = a;
        k.k1[i] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ U4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys &k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t h0, l0, h1, l1;
        mul_hi_lo(M0, c0, h0, l0);
        mul_hi_lo(M1, c2, h1, l1);
        const uint32_t n0 = h1 ^ c1 ^ k.k0[i];
        const uint32_t n2 = h0 ^ c3 ^ k.k1[i];
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    return U4{c0, c1, c2, c3};
}

// Philox4x32-10 of the counter (c0, t, q, 0) for many c0 under one key, with what depends on
// t, q and the key alone worked out once (philox_lead): in round 1 the product of q and words
// 0 and 1, in round 2 the product of round 1's word 0, in round 3 word 3.  The output is
// philox4x32_10(c0, t, q, 0, key); a draw takes 36 multiplies instead of 40.
struct PhiloxLead {
    uint32_t x0_2;  // round 2: word 0 = mulhi(M1, word 2) ^ x0_2
    uint32_t x2_2;  // round 2: word 2 = word 3 ^ x2_2
    uint32_t x2_3;  // round 3: word 2 = mulhi(M0, word 0) ^ x2_3
};

__host__ __device__ inline PhiloxLead philox_lead(uint32_t t, uint32_t q, const PhiloxKeys &k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint64_t p1 = (uint64_t)M1 * q;
    const uint32_t w0 = (uint32_t)(p1 >> 32) ^ t ^ k.k0[0], w1 = (uint32_t)p1;  // round 1, words 0 and 1
    const uint64_t p0 = (uint64_t)M0 * w0;                                       // round 2's product of word 0
    PhiloxLead ld;
    ld.x0_2 = w1 ^ k.k0[1];
    ld.x2_2 = (uint32_t)(p0 >> 32) ^ k.k1[1];
    ld.x2_3 = (uint32_t)p0 ^ k.k1[2];  // round 2's word 3 meets round 3's key word
    return ld;
}

__host__ __device__ __forceinline__ U4 philox4x32_10_lead(uint32_t c0, const PhiloxLead &ld, const PhiloxKeys &k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t h0, l0, h1, l1;
    mul_hi_lo(M0, c0, h0, l0);  // round 1: words 2 and 3
    const uint32_t a2 = h0 ^ k.k1[0], a3 = l0;
    mul_hi_lo(M1, a2, h1, l1);  // round 2: words 0, 1, 2 (word 3 is a constant)
    const uint32_t b0 = h1 ^ ld.x0_2, b1 = l1, b2 = a3 ^ ld.x2_2;
    mul_hi_lo(M0, b0, h0, l0);  // round 3
    mul_hi_lo(M1, b2, h1, l1);
    c0 = h1 ^ b1 ^ k.k0[2];
    uint32_t c1 = l1, c2 = h0 ^ ld.x2_3, c3 = l0;
#pragma unroll
    for (int i = 3; i < 10; ++i) {
        mul_hi_lo(M0, c0, h0, l0);
        mul_hi_lo(M1, c2, h1, l1);
        const uint32_t n0 = h1 ^ c1 ^ k.k0[i];
        const uint32_t n2 = h0 ^ c3 ^ k.k1[i];
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    return U4{c0, c1, c2, c3};
}

__host__ __device__ __forceinline__ uint32_t pick(const U4 &o, int i)
{
    return i == 0 ? o.x : (i == 1 ? o.y : (i == 2 ? o.z : o.w));
}

// Random bits of storage word sw (bit b = the bit of the word's site b) for `phase`
// (q for the zero-energy decision of sweep t, 2+q for the initial state, t = 0).
__device__ __forceinline__ uint32_t rng_word(const Geom &g, int64_t sw, uint32_t t, uint32_t phase,
                                             uint64_t S)
{
    const uint32_t k0 = (uint32_t)S, k1 = (uint32_t)(S >> 32);
    if (g.L >= 64) {
        const U4 o = philox4x32_10((uint32_t)(sw >> 2), t, phase, 0u, k0, k1);
        return pick(o, (int)(sw & 3));
    }
    const int64_t h0 = (int64_t)g.RB * sw;  // first compressed index of the row
    const int64_t w = h0 >> 5;
    const U4 o = philox4x32_10((uint32_t)(w >> 2), t, phase, 0u, k0, k1);
    return (pick(o, (int)(w & 3)) >> (h0 & 31)) & row_mask(g.RB);
}

// ---------------------------------------------------------------------------------
// Six-input bit-sliced counter: for each bit lane, u = number of set inputs among
// a..f.  Returns ge4 = [u >= 4] and eq3 = [u == 3] lane masks.
//   Two full adders give u = s1 + s2 + 2(c1 + c2); with a0 = s1^s2, a1 = s1&s2:
//   u = a0 + 2(a1 + c1 + c2).  u >= 4 <=> a1 + c1 + c2 >= 2 (majority);
//   u == 3 <=> a0 = 1 (then a1 = 0) and c1 + c2 = 1.
__device__ __forceinline__ void count6(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e,
                                       uint32_t f, uint32_t &ge4, uint32_t &eq3)
{
    const uint32_t s1 = a ^ b ^ c;
    const uint32_t c1 = (a & b) | (c & (a ^ b));
    const uint32_t s2 = d ^ e ^ f;
    const uint32_t c2 = (d & e) | (f & (d ^ e));
    const uint32_t a0 = s1 ^ s2;
    const uint32_t a1 = s1 & s2;
    ge4 = (a1 & c1) | (a1 & c2) | (c1 & c2);
    eq3 = a0 & (c1 ^ c2);
}

// New spins of one word (T -> 0 Glauber, Eq. 6): up where u >= 4, down where u <= 2,
// ties resolved by the rule: GLAUBER flips where the random bit is 1.
template <int RULE>
__device__ __forceinline__ uint32_t resolve(uint32_t s, uint32_t ge4, uint32_t eq3, uint32_t rnd)
{
    uint32_t tie;
    if (RULE == TIE_GLAUBER)
        tie = s ^ rnd;
    else if (RULE == TIE_ALWAYS)
        tie = ~s;
    else
        tie = s;
    return ge4 | (eq3 & tie);
}

// Programmatic dependent launch (a kernel launched with the programmatic stream
// serialisation attribute may be scheduled while the previous kernel of its stream drains):
// wait until the previous grid has completed and its memory operations are visible, then let
// the next grid of the stream start its own launch.  Executed first, before any access to
// global memory, so the kernel sees exactly what an ordinary stream order would give it;
// without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch attribute of the kernels that begin with pdl_enter().
inline cudaLaunchAttribute pdl_attribute()
{
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
    return a;
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a ^ b)); }

// New spins of the 128 sites of one uint4 (T -> 0 Glauber, Eq. 6).  With u the number of up
// neighbours and tau the tie bit (the old spin for the rule that never flips at zero energy,
// its complement for the rule that always flips, the old spin xor the random bit for Glauber),
// the new spin is [u + tau >= 4]: up where u >= 4, tau where u = 3, down where u <= 2.  Two
// full adders give u = s1 + s2 + 2 (c1 + c2); a third adds s1 + s2 + tau = s3 + 2 c3, so the
// new spin is the majority of c1, c2, c3.  Glauber draws Philox only where some site of the
// group has u = 3, i.e. s1 != s2 and c1 != c2.  For Glauber, COMPACT first reduces the adders
// to the masks [u >= 4] and [u = 3] (count6), which keeps two words per word live across the
// Philox call instead of four, at one more logic operation per word.
// LAZY (the default) draws Philox only for a group with a tie; without it every group draws
// (a warp draws whenever one of its 32 groups has a tie, which is nearly always, so the tie
// test then only costs instructions).
template <int RULE, bool COMPACT = true, bool LAZY = true>
__device__ __forceinline__ uint4 new_spins4(const uint4 &s, const uint4 &C, const uint4 &X, const uint4 &ym,
                                            const uint4 &yp, const uint4 &zm, const uint4 &zp, uint32_t group,
                                            uint32_t t, uint32_t q, const PhiloxKeys &keys)
{
    if (RULE == TIE_GLAUBER && COMPACT) {
        uint32_t g0, g1, g2, g3, e0, e1, e2, e3;
        count6(C.x, X.x, ym.x, yp.x, zm.x, zp.x, g0, e0);
        count6(C.y, X.y, ym.y, yp.y, zm.y, zp.y, g1, e1);
        count6(C.z, X.z, ym.z, yp.z, zm.z, zp.z, g2, e2);
        count6(C.w, X.w, ym.w, yp.w, zm.w, zp.w, g3, e3);
        U4 o{0u, 0u, 0u, 0u};
        if ((e0 | e1 | e2 | e3) != 0u) o = philox4x32_10_rk(group, t, q, 0u, keys);
        return make_uint4(resolve<RULE>(s.x, g0, e0, o.x), resolve<RULE>(s.y, g1, e1, o.y),
                          resolve<RULE>(s.z, g2, e2, o.z), resolve<RULE>(s.w, g3, e3, o.w));
    }
    const uint32_t s1x = C.x ^ X.x ^ ym.x, c1x = maj3(C.x, X.x, ym.x);
    const uint32_t s1y = C.y ^ X.y ^ ym.y, c1y = maj3(C.y, X.y, ym.y);
    const uint32_t s1z = C.z ^ X.z ^ ym.z, c1z = maj3(C.z, X.z, ym.z);
    const uint32_t s1w = C.w ^ X.w ^ ym.w, c1w = maj3(C.w, X.w, ym.w);
    const uint32_t s2x = yp.x ^ zm.x ^ zp.x, c2x = maj3(yp.x, zm.x, zp.x);
    const uint32_t s2y = yp.y ^ zm.y ^ zp.y, c2y = maj3(yp.y, zm.y, zp.y);
    const uint32_t s2z = yp.z ^ zm.z ^ zp.z, c2z = maj3(yp.z, zm.z, zp.z);
    const uint32_t s2w = yp.w ^ zm.w ^ zp.w, c2w = maj3(yp.w, zm.w, zp.w);
    uint4 tau;
    if (RULE == TIE_GLAUBER) {
        U4 o{0u, 0u, 0u, 0u};
        if (LAZY) {
            const uint32_t tie = ((s1x ^ s2x) & (c1x ^ c2x)) | ((s1y ^ s2y) & (c1y ^ c2y)) |
                                 ((s1z ^ s2z) & (c1z ^ c2z)) | ((s1w ^ s2w) & (c1w ^ c2w));
            if (tie != 0u) o = philox4x32_10_rk(group, t, q, 0u, keys);
        } else {
            o = philox4x32_10_rk(group, t, q, 0u, keys);
        }
        tau = make_uint4(s.x ^ o.x, s.y ^ o.y, s.z ^ o.z, s.w ^ o.w);
    } else if (RULE == TIE_ALWAYS) {
        tau = make_uint4(~s.x, ~s.y, ~s.z, ~s.w);
    } else {
        tau = s;
    }
    return make_uint4(maj3(c1x, c2x, maj3(s1x, s2x, tau.x)), maj3(c1y, c2y, maj3(s1y, s2y, tau.y)),
                      maj3(c1z, c2z, maj3(s1z, s2z, tau.z)), maj3(c1w, c2w, maj3(s1w, s2w, tau.w)));
}

// Neighbour words of storage word sw of sublattice q, read from the other sublattice
// array O.  X is the x-neighbour that is not at the same k (k-1 for p = 0, k+1 for
// p = 1; the other x-neighbour is C itself), Ym/Yp/Zm/Zp are the rows y-1, y+1,
// z-1, z+1 of O at the same word (their sites share x with ours).
struct Nbrs {
    uint32_t C, X, Ym, Yp, Zm, Zp;
};

__device__ __forceinline__ Nbrs load_nbrs(const uint32_t *__restrict__ O, const Geom &g, int64_t sw, int q)
{
    const int L = g.L, W = g.W;
    const int64_t row = sw / W;
    const int kw = (int)(sw - row * W);
    const int y = (int)(row % L);
    const int z = (int)(row / L);
    const int p = (y + z + q) & 1;
    Nbrs n;
    n.C = __ldg(O + sw);
    if (W >= 2) {
        if (p == 0) {
            const uint32_t e = __ldg(O + row * W + (kw == 0 ? W - 1 : kw - 1));
            n.X = (n.C << 1) | (e >> 31);
        } else {
            const uint32_t e = __ldg(O + row * W + (kw == W - 1 ? 0 : kw + 1));
            n.X = (n.C >> 1) | (e << 31);
        }
    } else {
        const int RB = g.RB;
        if (p == 0)
            n.X = ((n.C << 1) | (n.C >> (RB - 1))) & row_mask(RB);
        else
            n.X = (n.C >> 1) | ((n.C & 1u) << (RB - 1));
    }
    const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
    n.Ym = __ldg(O + ((int64_t)z * L + ym) * W + kw);
    n.Yp = __ldg(O + ((int64_t)z * L + yp) * W + kw);
    n.Zm = __ldg(O + ((int64_t)zm * L + y) * W + kw);
    n.Zp = __ldg(O + ((int64_t)zp * L + y) * W + kw);
    return n;
}

}  // namespace ising
