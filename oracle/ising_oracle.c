/*
 * CPU oracle for the zero-temperature checkerboard quench of the d=3 Ising model
 * (Gessert, Christiansen, Janke, "Superdiffusion-like behavior in zero-temperature
 * coarsening of the d=3 Ising model", arXiv:2305.12161).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA
 * library is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs may load it.  It shares no code, header,
 * table or helper with the CUDA library: everything below is written out from the
 * paper's definitions and from the published Philox4x32-10 generator.
 *
 * Representation: one signed byte per spin, s in {-1,+1}, site (x,y,z) in [0,L)^3 with
 * periodic boundaries, linear index i = x + L*(y + L*z) (64-bit: N = 2^33 at L = 2048).
 *
 * Every function is pinned by tests in tests/test_oracle_*.py (closed forms, fixed
 * points, brute-force recounts, known-answer vectors); see the per-function notes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TIE_GLAUBER 0 /* Eq. (6): a zero-energy flip is accepted with probability 1/2 */
#define ORC_TIE_ALWAYS 1  /* T->0 limit of Metropolis, min(1, e^0) = 1 (Supp. Methods I B) */
#define ORC_TIE_NEVER 2   /* zero-energy flips rejected */

/* Host threads used by the OpenMP loops below (1 when built without OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as easy
 * as 1, 2, 3").  A 4x32-bit counter and a 2x32-bit key; ten rounds.  Each round
 * multiplies counter words 0 and 2 by the two round multipliers into 64-bit products,
 * recombines hi/lo halves with words 1 and 3 and the round key, and then the key is
 * bumped by the two Weyl constants (golden ratio and sqrt(3)-1 in 32-bit fixed point).
 * Pinned by the published known-answer vectors (tests/golden/philox4x32_10_kat.txt)
 * and by an independent library implementation. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------------ */
/* Random-bit addressing.  The paper names no generator and no mapping from random
 * numbers to sites; this library fixes one so that every run is reproducible:
 *   - a site (x,y,z) of sublattice q = (x+y+z) mod 2 gets the compressed index
 *       h = (x >> 1) + (L/2) * (y + L*z)            in [0, N/2),
 *     its 32-bit word w = h >> 5 and its bit j = h & 31;
 *   - key = (lo32(S), hi32(S)) with S = seed + replica (mod 2^64);
 *   - counter = (w >> 2, t, phase, 0), phase = q for the update of sweep t (0-based),
 *     phase = 2 + q for the T = infinity initial state (t = 0);
 *   - the bit is bit j of output word (w & 3). */
int orc_rng_bit(uint64_t S, uint32_t t, uint32_t phase, int64_t h)
{
    int64_t w = h >> 5;
    int j = (int)(h & 31);
    uint32_t ctr[4] = {(uint32_t)(w >> 2), t, phase, 0u};
    uint32_t key[2] = {(uint32_t)(S & 0xffffffffu), (uint32_t)(S >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return (int)((o[w & 3] >> j) & 1u);
}

static inline int64_t site(int64_t L, int64_t x, int64_t y, int64_t z)
{
    return x + L * (y + L * z);
}

static inline int64_t wrap(int64_t a, int64_t L) { return ((a % L) + L) % L; }

static inline int64_t compressed_index(int64_t L, int64_t x, int64_t y, int64_t z)
{
    return (x >> 1) + (L / 2) * (y + L * z);
}

/* ------------------------------------------------------------------------------ */
/* T = infinity initial state (Results and Discussion: random spin configurations with
 * m ~ 0): every spin is +1 or -1 independently with probability 1/2, the bit drawn
 * with phase 2 + q at t = 0. */
void orc_init(int L_, uint64_t S, int8_t *s)
{
    const int64_t L = L_;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                int q = (int)((x + y + z) & 1);
                int b = orc_rng_bit(S, 0u, (uint32_t)(2 + q), compressed_index(L, x, y, z));
                s[site(L, x, y, z)] = b ? (int8_t)1 : (int8_t)-1;
            }
}

/* ------------------------------------------------------------------------------ */
/* One half-sweep of the checkerboard update (Methods, "Checkerboard update"): every
 * site of sublattice q (sites with (x+y+z) mod 2 == q; the 3-d generalisation of the
 * checkerboard figure) is proposed once, all of them at the same time.  Their six
 * nearest neighbours all lie on the other sublattice, so every proposal sees the
 * neighbour values from before this half-sweep.
 *
 * Acceptance is the T -> 0 Glauber rule, Eq. (6): with H = -sum_<ij> s_i s_j (J = 1),
 * flipping s_i changes the energy by dE = 2 s_i sum_nn s_j = 2 s_i (2u - 6), u = number
 * of up neighbours.  dE < 0 -> flip, dE > 0 -> keep, dE = 0 (u = 3) -> flip with
 * probability 1/2, i.e. when the site's random bit is 1 (or per the rule flag).
 * Therefore the new spin is up for u >= 4 and down for u <= 2.
 *
 * Returns the number of flips; *dB receives the change of the broken-bond count B
 * accumulated flip by flip (a flipped site with a aligned neighbours before the flip
 * changes B by 2a - 6), *dM the change of the magnetisation. */
/* New value of site (x,y,z) of sublattice q under the rule above, reading its six
 * neighbours from s; *aligned receives the number of neighbours equal to the old spin. */
static int8_t site_new_value(int64_t L, const int8_t *s, int64_t x, int64_t y, int64_t z, int q, uint32_t t,
                             uint64_t S, int rule, int *aligned)
{
    int8_t nb[6] = {
        s[site(L, wrap(x + 1, L), y, z)], s[site(L, wrap(x - 1, L), y, z)],
        s[site(L, x, wrap(y + 1, L), z)], s[site(L, x, wrap(y - 1, L), z)],
        s[site(L, x, y, wrap(z + 1, L))], s[site(L, x, y, wrap(z - 1, L))]};
    int u = 0;
    for (int k = 0; k < 6; ++k) u += (nb[k] == 1);
    int8_t old = s[site(L, x, y, z)];
    int a = 0;
    for (int k = 0; k < 6; ++k) a += (nb[k] == old);
    if (aligned) *aligned = a;
    if (u >= 4) return 1;
    if (u <= 2) return -1;
    if (rule == ORC_TIE_ALWAYS) return (int8_t)-old;
    if (rule == ORC_TIE_NEVER) return old;
    int r = orc_rng_bit(S, t, (uint32_t)q, compressed_index(L, x, y, z));
    return r ? (int8_t)-old : old;
}

int64_t orc_half_sweep(int L_, int8_t *s, int q, uint32_t t, uint64_t S, int rule,
                       int64_t *dB, int64_t *dM)
{
    const int64_t L = L_;
    int64_t flips = 0, db = 0, dm = 0;
#pragma omp parallel for schedule(static) reduction(+ : flips, db, dm)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != q) continue;
                int aligned = 0;
                int8_t old = s[site(L, x, y, z)];
                int8_t nw = site_new_value(L, s, x, y, z, q, t, S, rule, &aligned);
                if (nw != old) {
                    flips += 1;
                    db += 2 * aligned - 6;
                    dm += (int64_t)nw - (int64_t)old;
                    s[site(L, x, y, z)] = nw;
                }
            }
    if (dB) *dB = db;
    if (dM) *dM = dm;
    return flips;
}

/* The values that the half-sweep of sublattice q at sweep t would give the n listed
 * sites (linear indices, each on sublattice q), without modifying s.  A site's update
 * reads only the other sublattice, so this equals the full half-sweep at those sites;
 * it lets lattices too large for a full oracle pass be checked site by site. */
void orc_update_sites(int L_, const int8_t *s, int q, uint32_t t, uint64_t S, int rule,
                      const int64_t *sites, int64_t n, int8_t *out)
{
    const int64_t L = L_;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = sites[k];
        int64_t x = i % L, y = (i / L) % L, z = i / (L * L);
        out[k] = site_new_value(L, s, x, y, z, q, t, S, rule, NULL);
    }
}

/* n Monte Carlo sweeps starting at completed-sweep count t0.  One MCS (Methods,
 * "Random-site-flip update": N proposals) is the red (q = 0) half-sweep followed by
 * the blue (q = 1) half-sweep, both with the sweep's 0-based index as counter word. */
void orc_sweeps(int L, int8_t *s, uint32_t t0, int64_t n, uint64_t S, int rule)
{
    for (int64_t k = 0; k < n; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        orc_half_sweep(L, s, 0, t, S, rule, NULL, NULL);
        orc_half_sweep(L, s, 1, t, S, rule, NULL, NULL);
    }
}

/* ------------------------------------------------------------------------------ */
/* Integer observables of one configuration, written as a record
 *   rec[0] = t, rec[1] = M = sum_i s_i, rec[2] = B = number of unequal nearest-
 *   neighbour pairs, then D_x(r), D_y(r), D_z(r) for r = 0..L/2, with
 *   D_a(r) = #{ i : s_i != s_(i + r e_a) }.
 * The spin-spin sum of Eq. (2) along axis a follows as sum_i s_i s_(i+r e_a) =
 * N - 2 D_a(r); the energy of H = -sum_<ij> s_i s_j is E = -(3N - 2B). */
int64_t orc_record_len(int L) { return 3 + 3 * (int64_t)(L / 2 + 1); }

/* M and B of one configuration. */
void orc_magnetisation_bonds(int L_, const int8_t *s, int64_t *M_out, int64_t *B_out)
{
    const int64_t L = L_;
    int64_t M = 0, B = 0;
#pragma omp parallel for schedule(static) reduction(+ : M, B)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                int8_t v = s[site(L, x, y, z)];
                M += v;
                B += (v != s[site(L, wrap(x + 1, L), y, z)]);
                B += (v != s[site(L, x, wrap(y + 1, L), z)]);
                B += (v != s[site(L, x, y, wrap(z + 1, L))]);
            }
    *M_out = M;
    *B_out = B;
}

/* D_x(r), D_y(r), D_z(r) for one distance r. */
void orc_corr_lag(int L_, const int8_t *s, int64_t r, int64_t *D3)
{
    const int64_t L = L_;
    int64_t dx = 0, dy = 0, dz = 0;
#pragma omp parallel for schedule(static) reduction(+ : dx, dy, dz)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                int8_t v = s[site(L, x, y, z)];
                dx += (v != s[site(L, wrap(x + r, L), y, z)]);
                dy += (v != s[site(L, x, wrap(y + r, L), z)]);
                dz += (v != s[site(L, x, y, wrap(z + r, L))]);
            }
    D3[0] = dx;
    D3[1] = dy;
    D3[2] = dz;
}

/* D_x(r), D_y(r), D_z(r) for the n distances lags[0..n), each in [0, L), written to
 * D3[3j + a].  Same definition as orc_corr_lag, counted line by line: the L sites of one
 * periodic line along axis a are copied twice in a row into a buffer, so that the
 * partner of position k at distance r is buffer entry k + r, and every lag is one pass
 * over the buffer.  A second, independent way of counting Eq. (2)'s pairs: the tests
 * require it to equal orc_corr_lag at every lag on small lattices. */
void orc_corr_lags(int L_, const int8_t *s, const int64_t *lags, int64_t n, int64_t *D3)
{
    const int64_t L = L_;
    for (int64_t k = 0; k < 3 * n; ++k) D3[k] = 0;
    for (int a = 0; a < 3; ++a) {
        /* step along the line, and the steps of the two coordinates that fix the line
         * (the faster one first, so that consecutive lines share cache lines) */
        const int64_t sa = a == 0 ? 1 : (a == 1 ? L : L * L);
        const int64_t su = a == 0 ? L : 1;
        const int64_t sv = a == 2 ? L : L * L;
#pragma omp parallel
        {
            int8_t *ln = (int8_t *)malloc((size_t)(2 * L));
            int64_t *acc = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
#pragma omp for schedule(static)
            for (int64_t line = 0; line < L * L; ++line) {
                const int64_t base = (line % L) * su + (line / L) * sv;
                for (int64_t k = 0; k < L; ++k) {
                    ln[k] = s[base + k * sa];
                    ln[L + k] = ln[k];
                }
                for (int64_t j = 0; j < n; ++j) {
                    const int8_t *p = ln + lags[j];
                    int32_t c = 0;
                    for (int64_t k = 0; k < L; ++k) c += (ln[k] != p[k]);
                    acc[j] += c;
                }
            }
#pragma omp critical
            for (int64_t j = 0; j < n; ++j) D3[3 * j + a] += acc[j];
            free(ln);
            free(acc);
        }
    }
}

void orc_record(int L_, const int8_t *s, int64_t t, int64_t *rec)
{
    const int64_t L = L_;
    const int64_t R = L / 2;
    rec[0] = t;
    orc_magnetisation_bonds(L_, s, &rec[1], &rec[2]);
    int64_t *lags = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R + 1));
    int64_t *D3 = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(R + 1));
    for (int64_t r = 0; r <= R; ++r) lags[r] = r;
    orc_corr_lags(L_, s, lags, R + 1, D3);
    int64_t *Dx = rec + 3, *Dy = rec + 3 + (R + 1), *Dz = rec + 3 + 2 * (R + 1);
    for (int64_t r = 0; r <= R; ++r) {
        Dx[r] = D3[3 * r + 0];
        Dy[r] = D3[3 * r + 1];
        Dz[r] = D3[3 * r + 2];
    }
    free(D3);
    free(lags);
}

/* ------------------------------------------------------------------------------ */
/* Quantities derived from one record (double precision):
 *   out[0] = e   = E/N = -3 + 2B/N          (energy per spin)
 *   out[1] = m   = M/N                      (magnetisation per spin)
 *   out[2] = l_E = N/B = 2/(e - e0), e0 = -3 (length from the excess energy; +inf if B=0)
 *   out[3] = l_C: C(r) = G(r)/(3N) with G(r) = sum_a (N - 2 D_a(r)) (minus m^2 when
 *            `connected`, the second term of Eq. (2) taken per sample); l_C is the
 *            intersection of C with the constant c (Results: "intersection of C(r,t)
 *            with a constant value of c = 0.5"), linearly interpolated at the first r0
 *            with C(r0) >= c > C(r0+1); NaN when C does not cross c for r <= L/2. */
void orc_derived(int L_, const int64_t *rec, double c, int connected, double *out)
{
    const int64_t L = L_;
    const int64_t R = L / 2;
    const double N = (double)L * (double)L * (double)L;
    const int64_t M = rec[1], B = rec[2];
    const int64_t *Dx = rec + 3, *Dy = rec + 3 + (R + 1), *Dz = rec + 3 + 2 * (R + 1);
    double m = (double)M / N;
    out[0] = -3.0 + 2.0 * (double)B / N;
    out[1] = m;
    out[2] = (B == 0) ? INFINITY : N / (double)B;
    double lc = NAN;
    double sub = connected ? m * m : 0.0;
    for (int64_t r = 0; r < R; ++r) {
        double g0 = (N - 2.0 * (double)Dx[r]) + (N - 2.0 * (double)Dy[r]) + (N - 2.0 * (double)Dz[r]);
        double g1 = (N - 2.0 * (double)Dx[r + 1]) + (N - 2.0 * (double)Dy[r + 1]) +
                    (N - 2.0 * (double)Dz[r + 1]);
        double c0 = g0 / (3.0 * N) - sub;
        double c1 = g1 / (3.0 * N) - sub;
        if (c0 >= c && c > c1) {
            lc = (double)r + (c0 - c) / (c0 - c1);
            break;
        }
    }
    out[3] = lc;
}

/* ------------------------------------------------------------------------------ */
/* Menger-sponge initial state (Results, the sponge test: the lattice is tiled with
 * k-th-iteration Menger sponges of side 3^k, each drawn in up or down spins at random).
 * Reading used here: a cell (a,b,c) of a tile, 0 <= a,b,c < 3^k, belongs to the sponge
 * unless at some base-3 digit position at least two of its three digits equal 1 (the
 * centre and face-centre sub-cubes removed at every level); the sponge's cells take the
 * tile's sign sigma, the removed cells take -sigma.  Tiles are cut at the lattice edge when
 * 3^k does not divide L.  Tile T = tx + nT*(ty + nT*tz), nT = ceil(L/3^k), gets sigma = +1
 * when bit (T & 31) of word ((T >> 5) & 3) of Philox(counter (T >> 7, 0, 4, 0), key S) is 1. */
int orc_menger_member(int64_t a, int64_t b, int64_t c, int k)
{
    for (int d = 0; d < k; ++d) {
        int ones = (a % 3 == 1) + (b % 3 == 1) + (c % 3 == 1);
        if (ones >= 2) return 0;
        a /= 3;
        b /= 3;
        c /= 3;
    }
    return 1;
}

int orc_menger_tile_sign(uint64_t S, int64_t T)
{
    uint32_t ctr[4] = {(uint32_t)(T >> 7), 0u, 4u, 0u};
    uint32_t key[2] = {(uint32_t)(S & 0xffffffffu), (uint32_t)(S >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return ((o[(T >> 5) & 3] >> (T & 31)) & 1u) ? 1 : -1;
}

void orc_init_menger(int L_, uint64_t S, int k, int8_t *s)
{
    const int64_t L = L_;
    int64_t side = 1;
    for (int d = 0; d < k; ++d) side *= 3;
    const int64_t nT = (L + side - 1) / side;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                int64_t T = x / side + nT * (y / side + nT * (z / side));
                int sigma = orc_menger_tile_sign(S, T);
                int in = orc_menger_member(x % side, y % side, z % side, k);
                s[site(L, x, y, z)] = (int8_t)(in ? sigma : -sigma);
            }
}

/* ------------------------------------------------------------------------------ */
/* Mixed cycle (Supp. Methods I B: the sublattice updated first is chosen at random in
 * every sweep, which restores detailed balance).  Sweep t updates blue (q = 1) first when
 * bit 0 of word 0 of Philox(counter (0, t, 5, 0), key S) is 1, otherwise red first. */
int orc_mixed_order(uint64_t S, uint32_t t)
{
    uint32_t ctr[4] = {0u, t, 5u, 0u};
    uint32_t key[2] = {(uint32_t)(S & 0xffffffffu), (uint32_t)(S >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return (int)(o[0] & 1u);
}

void orc_sweeps_mixed(int L, int8_t *s, uint32_t t0, int64_t n, uint64_t S, int rule)
{
    for (int64_t k = 0; k < n; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        int first = orc_mixed_order(S, t);
        orc_half_sweep(L, s, first, t, S, rule, NULL, NULL);
        orc_half_sweep(L, s, 1 - first, t, S, rule, NULL, NULL);
    }
}

/* ------------------------------------------------------------------------------ */
/* Random-site-flip (rsf) update (Methods, "Random-site-flip update"): one MC step picks a
 * site uniformly at random and proposes to flip it; the flip is accepted with Eq. (6) at
 * T -> 0 (always if dE < 0, never if dE > 0, with probability 1/2 if dE = 0, or per the
 * rule flag); N = L^3 steps are one MCS.  The steps are sequential: each one sees every
 * flip before it, and within a sweep a site may be proposed several times or not at all.
 * This is the paper's baseline dynamics, against which the checkerboard's time is
 * rescaled (Supplementary Table of time factors: checkerboard 1.75, rsf 1).
 *
 * Random numbers (the paper names no generator): step k (0 <= k < N) of sweep t (0-based)
 * takes one Philox4x32-10 call with counter (lo32 k, t, 7, hi32 k) and key (lo32 S, hi32 S);
 * the site is the 64-bit integer o[1]:o[0] modulo N (bias at most N / 2^64) and the
 * zero-energy decision is bit 0 of o[2]. */
void orc_rsf_draw(uint64_t S, uint32_t t, int64_t k, int64_t N, int64_t *site_out, int *bit_out)
{
    uint32_t ctr[4] = {(uint32_t)((uint64_t)k & 0xffffffffu), t, 7u, (uint32_t)((uint64_t)k >> 32)};
    uint32_t key[2] = {(uint32_t)(S & 0xffffffffu), (uint32_t)(S >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    const uint64_t r = ((uint64_t)o[1] << 32) | (uint64_t)o[0];
    *site_out = (int64_t)(r % (uint64_t)N);
    *bit_out = (int)(o[2] & 1u);
}

/* n rsf sweeps in place from completed-sweep count t0.  Returns the number of accepted
 * flips; *dB receives the change of the broken-bond count accumulated flip by flip (a
 * flipped site with a aligned neighbours before the flip changes B by 2a - 6), *dM that
 * of the magnetisation. */
int64_t orc_sweeps_rsf(int L_, int8_t *s, uint32_t t0, int64_t n, uint64_t S, int rule, int64_t *dB, int64_t *dM)
{
    const int64_t L = L_;
    const int64_t N = L * L * L;
    int64_t flips = 0, db = 0, dm = 0;
    for (int64_t sweep = 0; sweep < n; ++sweep) {
        const uint32_t t = t0 + (uint32_t)sweep;
        for (int64_t k = 0; k < N; ++k) {
            int64_t i;
            int bit;
            orc_rsf_draw(S, t, k, N, &i, &bit);
            const int64_t x = i % L, y = (i / L) % L, z = i / (L * L);
            const int8_t nb[6] = {
                s[site(L, wrap(x + 1, L), y, z)], s[site(L, wrap(x - 1, L), y, z)],
                s[site(L, x, wrap(y + 1, L), z)], s[site(L, x, wrap(y - 1, L), z)],
                s[site(L, x, y, wrap(z + 1, L))], s[site(L, x, y, wrap(z - 1, L))]};
            const int8_t old = s[i];
            int u = 0, a = 0;
            for (int j = 0; j < 6; ++j) {
                u += (nb[j] == 1);
                a += (nb[j] == old);
            }
            /* dE = 2 old (2u - 6): accept for dE < 0, reject for dE > 0, tie at u = 3 */
            int8_t nw;
            if (u >= 4)
                nw = 1;
            else if (u <= 2)
                nw = -1;
            else if (rule == ORC_TIE_ALWAYS)
                nw = (int8_t)-old;
            else if (rule == ORC_TIE_NEVER)
                nw = old;
            else
                nw = bit ? (int8_t)-old : old;
            if (nw != old) {
                s[i] = nw;
                flips += 1;
                db += 2 * a - 6;
                dm += (int64_t)nw - (int64_t)old;
            }
        }
    }
    if (dB) *dB = db;
    if (dM) *dM = dm;
    return flips;
}

/* ------------------------------------------------------------------------------ */
/* Double-checkerboard update (Supp. Methods I A: Weigel's GPU domain decomposition,
 * generalised to d = 3).  The lattice is cut into blocks of bx*by*bz sites; block
 * (i, j, k) = (x / bx, y / by, z / bz) is red (colour 0) when i + j + k is even and blue
 * (colour 1) otherwise.  With an even number of blocks along every axis that is cut (or a
 * single block spanning the axis), two blocks of one colour never share a face, so all
 * blocks of a colour can be updated at once.  One sweep: for each colour in turn, every
 * block of that colour updates its sites of one fine sublattice (parity of x + y + z) all
 * at once, and then the sites of the other parity; sites in other blocks keep their values
 * during that colour's pass.
 *
 * 01 cycle (the steps listed in I A): red blocks first, and in every block the sites of
 * odd parity first (the darker sites of the paper's 2-d example figure are those with
 * x + y odd).  Mixed cycle (I B): the first colour is drawn once per sweep with
 * orc_mixed_order (blue first when it is 1), and the first fine sublattice independently
 * for every block and sweep: block beta = i + nbx*(j + nby*k) starts with the sites of
 * parity 1 when bit (beta & 31) of word ((beta >> 5) & 3) of
 * Philox(counter (beta >> 7, t, 6, 0), key S) is 1, else with those of parity 0.
 * A site's zero-energy decision uses the same random bit as in the checkerboard update
 * (phase = its parity, counter word = its compressed index), so the schemes differ only
 * in the order in which the proposals are made. */
int orc_dcb_valid(int L, int bx, int by, int bz)
{
    const int b[3] = {bx, by, bz};
    if (L < 2 || (L & 1)) return 0;
    for (int a = 0; a < 3; ++a) {
        if (b[a] < 1 || L % b[a] != 0) return 0;
        const int nb = L / b[a];
        if (nb != 1 && (nb & 1)) return 0;
    }
    return 1;
}

int orc_dcb_fine_first(uint64_t S, uint32_t t, int64_t beta)
{
    uint32_t ctr[4] = {(uint32_t)(beta >> 7), t, 6u, 0u};
    uint32_t key[2] = {(uint32_t)(S & 0xffffffffu), (uint32_t)(S >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return (int)((o[(beta >> 5) & 3] >> (beta & 31)) & 1u);
}

/* Every site of parity q inside the block with corner (x0, y0, z0), proposed once.  The
 * sites of one parity are not neighbours of one another, so updating them one after the
 * other in place gives the same result as updating them all at once. */
static void dcb_block_pass(int64_t L, int8_t *s, int64_t x0, int64_t y0, int64_t z0, int64_t bx, int64_t by,
                           int64_t bz, int q, uint32_t t, uint64_t S, int rule)
{
    for (int64_t z = z0; z < z0 + bz; ++z)
        for (int64_t y = y0; y < y0 + by; ++y)
            for (int64_t x = x0; x < x0 + bx; ++x) {
                if (((x + y + z) & 1) != q) continue;
                s[site(L, x, y, z)] = site_new_value(L, s, x, y, z, q, t, S, rule, NULL);
            }
}

int orc_sweeps_dcb(int L_, int8_t *s, uint32_t t0, int64_t n, uint64_t S, int rule, int bx, int by, int bz,
                   int mixed)
{
    if (!orc_dcb_valid(L_, bx, by, bz)) return -1;
    const int64_t L = L_;
    const int64_t nbx = L / bx, nby = L / by, nbz = L / bz;
    const int64_t nblocks = nbx * nby * nbz;
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t t = t0 + (uint32_t)k;
        const int first = mixed ? orc_mixed_order(S, t) : 0;
        for (int pass = 0; pass < 2; ++pass) {
            const int colour = first ^ pass;
#pragma omp parallel for schedule(dynamic, 1)
            for (int64_t beta = 0; beta < nblocks; ++beta) {
                const int64_t i = beta % nbx, j = (beta / nbx) % nby, kk = beta / (nbx * nby);
                if (((i + j + kk) & 1) != colour) continue;
                const int f0 = mixed ? orc_dcb_fine_first(S, t, beta) : 1;
                dcb_block_pass(L, s, i * bx, j * by, kk * bz, bx, by, bz, f0, t, S, rule);
                dcb_block_pass(L, s, i * bx, j * by, kk * bz, bx, by, bz, 1 - f0, t, S, rule);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Three-dimensional correlation and structure factor, radially averaged (Methods,
 * "Calculating the correlation function": the paper obtains the spin-spin sum for every
 * lag vector from an FFT, Eq. (3), and averages it radially; Results: S(k,t) is the
 * Fourier transform of C).  Written out here from the definitions, by brute force.
 *
 * Lag and mode vectors: each component j in [0, L) stands for its minimal image
 * d = j for j <= L/2, j - L otherwise (|d| = L/2 for j = L/2 either way).
 * Radial bin of a vector with squared length D: b = round(sqrt(D)), computed exactly in
 * integers as (isqrt(4D) + 1) / 2 (sqrt(D) + 1/2 is never an integer for integer D, so no
 * vector sits on a bin edge).  Bins b = 0 .. nbins-1, nbins = (isqrt(3 L^2) + 1)/2 + 1;
 * bins beyond L/2 are cut by the cube's corners. */
int64_t orc_isqrt(int64_t n)
{
    if (n <= 0) return 0;
    int64_t lo = 0, hi = 1;
    while (hi * hi <= n) hi *= 2;
    while (hi - lo > 1) {  /* invariant: lo^2 <= n < hi^2 */
        const int64_t mid = lo + (hi - lo) / 2;
        if (mid * mid <= n) lo = mid; else hi = mid;
    }
    return lo;
}

static inline int64_t min_image(int64_t j, int64_t L) { return j <= L / 2 ? j : j - L; }

int64_t orc_radial_bin(int L_, int64_t x, int64_t y, int64_t z)
{
    const int64_t L = L_;
    const int64_t a = min_image(x, L), b = min_image(y, L), c = min_image(z, L);
    return (orc_isqrt(4 * (a * a + b * b + c * c)) + 1) / 2;
}

int64_t orc_radial_nbins(int L_)
{
    const int64_t L = L_;
    return (orc_isqrt(3 * L * L) + 1) / 2 + 1;
}

/* G(k) = sum_i s_i s_(i+k) for every lag k = (kx, ky, kz), stored at kx + L(ky + L kz):
 * the double sum of Eq. (2) over all pairs at that separation, O(N^2). */
void orc_corr3d(int L_, const int8_t *s, int64_t *G)
{
    const int64_t L = L_;
    const int64_t N = L * L * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < N; ++k) {
        const int64_t kx = k % L, ky = (k / L) % L, kz = k / (L * L);
        int64_t acc = 0;
        for (int64_t z = 0; z < L; ++z)
            for (int64_t y = 0; y < L; ++y)
                for (int64_t x = 0; x < L; ++x)
                    acc += (int64_t)s[site(L, x, y, z)] *
                           (int64_t)s[site(L, (x + kx) % L, (y + ky) % L, (z + kz) % L)];
        G[k] = acc;
    }
}

/* Radially averaged correlation C(r) = (1/n_r) sum_{k in bin r} G(k)/N and the number n_r
 * of lag vectors in each bin.  The integer sums of G over a bin are formed first and
 * divided once, C(r) = (double) sum_G / ((double) N * (double) n_r), so the value does not
 * depend on the order of summation. */
void orc_radial_corr(int L_, const int8_t *s, double *C, int64_t *count)
{
    const int64_t L = L_;
    const int64_t N = L * L * L;
    const int64_t nb = orc_radial_nbins(L_);
    int64_t *G = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *sumG = (int64_t *)calloc((size_t)nb, sizeof(int64_t));
    if (!G || !sumG) {
        free(G);
        free(sumG);
        return;
    }
    orc_corr3d(L_, s, G);
    for (int64_t b = 0; b < nb; ++b) count[b] = 0;
    for (int64_t k = 0; k < N; ++k) {
        const int64_t b = orc_radial_bin(L_, k % L, (k / L) % L, k / (L * L));
        sumG[b] += G[k];
        count[b] += 1;
    }
    for (int64_t b = 0; b < nb; ++b)
        C[b] = count[b] ? (double)sumG[b] / ((double)N * (double)count[b]) : 0.0;
    free(G);
    free(sumG);
}

/* Structure factor S(n) = |sum_x s_x exp(-2 pi i n.x / L)|^2 / N for every mode
 * n = (nx, ny, nz) (wave vector 2 pi n / L), by the direct O(N^2) sum, radially averaged
 * over the same bins as C (bin b is wave number 2 pi b / L).  The phase n.x mod L indexes a
 * table of the L complex roots of unity. */
void orc_structure_factor(int L_, const int8_t *s, double *S, int64_t *count)
{
    const int64_t L = L_;
    const int64_t N = L * L * L;
    const int64_t nb = orc_radial_nbins(L_);
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)L);
    double *P = (double *)malloc(sizeof(double) * (size_t)N);
    if (!cs || !P) {
        free(cs);
        free(P);
        return;
    }
    for (int64_t j = 0; j < L; ++j) {
        const double two_pi = 6.283185307179586476925286766559;
        cs[2 * j] = cos(two_pi * (double)j / (double)L);
        cs[2 * j + 1] = -sin(two_pi * (double)j / (double)L);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t n = 0; n < N; ++n) {
        const int64_t nx = n % L, ny = (n / L) % L, nz = n / (L * L);
        double re = 0.0, im = 0.0;
        for (int64_t z = 0; z < L; ++z)
            for (int64_t y = 0; y < L; ++y)
                for (int64_t x = 0; x < L; ++x) {
                    const int64_t ph = (nx * x + ny * y + nz * z) % L;
                    const double v = (double)s[site(L, x, y, z)];
                    re += v * cs[2 * ph];
                    im += v * cs[2 * ph + 1];
                }
        P[n] = (re * re + im * im) / (double)N;
    }
    for (int64_t b = 0; b < nb; ++b) {
        S[b] = 0.0;
        count[b] = 0;
    }
    for (int64_t n = 0; n < N; ++n) {
        const int64_t b = orc_radial_bin(L_, n % L, (n / L) % L, n / (L * L));
        S[b] += P[n];
        count[b] += 1;
    }
    for (int64_t b = 0; b < nb; ++b)
        if (count[b]) S[b] /= (double)count[b];
    free(cs);
    free(P);
}

/* Length from the radial C: the crossing rule of orc_derived applied to C(r) for
 * r = 0 .. L/2 (the shells that the cube contains whole): r0 + (C(r0) - c)/(C(r0) - C(r0+1))
 * at the first r0 < L/2 with C(r0) >= c > C(r0+1), NaN if none; `sub` is subtracted from C
 * first (m^2 for the connected variant). */
double orc_radial_length(int L_, const double *C, double c, double sub)
{
    const int64_t R = L_ / 2;
    for (int64_t r = 0; r < R; ++r) {
        const double c0 = C[r] - sub, c1 = C[r + 1] - sub;
        if (c0 >= c && c > c1) return (double)r + (c0 - c) / (c0 - c1);
    }
    return NAN;
}

/* G(k) = sum_i s_i s_(i+k) for the single lag vector k = (dx, dy, dz) (any integers, taken
 * modulo L): the same double sum as orc_corr3d for one k, so that lags can be checked at
 * lattice sizes where the full O(N^2) array is out of reach. */
int64_t orc_corr_vec(int L_, const int8_t *s, int64_t dx, int64_t dy, int64_t dz)
{
    const int64_t L = L_;
    const int64_t ox = wrap(dx, L), oy = wrap(dy, L), oz = wrap(dz, L);
    int64_t acc = 0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y) {
            const int8_t *a = s + site(L, 0, y, z);
            const int8_t *b = s + site(L, 0, (y + oy) % L, (z + oz) % L);
            for (int64_t x = 0; x < L; ++x) acc += (int64_t)a[x] * (int64_t)b[(x + ox) % L];
        }
    return acc;
}
