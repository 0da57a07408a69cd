/*
 * ising_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * checkerboard-Metropolis Ising model (2D square / 3D cubic lattice, J = 1,
 * h = 0, periodic boundaries).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA engine; the engine must
 * never call it.
 *
 * What it follows (Tomov et al., "Benchmarking and Implementation of
 * Probability-Based Simulations on Programmable Graphics Cards", 2003):
 *   - energy        E(S) = - sum over lattice edges <j,k> of S(j) S(k)   (Sec. 2.2)
 *   - magnetisation #up - #down = sum_j S(j)                              (Sec. 2.2)
 *   - random initial state: spin up with probability p                   (Sec. 2.2)
 *   - checkerboard colouring; a colour pass visits all sites of one
 *     colour, black pass then white pass                                  (Sec. 2.2)
 *   - Metropolis decision: dE < 0 accept; otherwise draw R in [0,1] and
 *     accept iff R <= exp(-dE/kT)                                         (Sec. 2.2)
 *   - expected value E(F) = sum_i F(S_i) P(S_i) with Boltzmann P          (Eq. 1)
 *
 * Readings where the paper is silent:
 *   - one "sweep" here is a black pass followed by a white pass, so every
 *     site is visited once per sweep; colour c(x,y[,z]) = (x+y[+z]) mod 2,
 *     black = colour 0;
 *   - beta = J/kT is dimensionless with J = 1, and dE = 2k where
 *     k = s_i * (sum of the 2*dims neighbours of i);
 *   - dE <= 0 always flips (R <= 1 holds for every draw); for dE > 0 the
 *     uniform R is a 32-bit integer u and the flip happens iff
 *     u < thr[k] = floor(exp(-2 beta k) * 2^32);
 *   - the paper's linear congruential generator (constants unstated) is
 *     replaced by Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by
 *     the 64-bit seed and counted by (site group, sweep, colour, tag), so
 *     that every draw is a pure function of (seed, sweep, site);
 *   - canonical site index i = x + L*y (+ L*L*z), half index hh = i >> 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the description in Salmon et al. (SC'11):    */
/* a 4-word counter is mixed by 10 rounds, each round multiplying words 0   */
/* and 2 by fixed odd constants, swapping the halves of the products into  */
/* the other lanes and xoring the round key in; the 2-word key is bumped by */
/* the Weyl constants (golden ratio, sqrt(3)-1) between rounds.              */
/* ------------------------------------------------------------------------ */

static const uint32_t PHILOX_MUL_A = 0xD2511F53u; /* multiplies counter word 0 */
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u; /* multiplies counter word 2 */
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t n0 = pb_hi ^ x1 ^ k0;
        uint32_t n1 = pb_lo;
        uint32_t n2 = pa_hi ^ x3 ^ k1;
        uint32_t n3 = pa_lo;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 32-bit uniform: word (w & 3) of Philox(key = seed, ctr). */
static uint32_t draw_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, unsigned w)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w & 3u];
}

/* Counter tags in word 3 keep the three uses of the stream disjoint. */
enum { TAG_SWEEP = 0, TAG_INIT = 1, TAG_SEQUENTIAL = 2 };

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds (Sec. 2.2, Metropolis step 4 with R -> u / 2^32):  */
/* thr[j] = floor(exp(-2 beta k) * 2^32) for k = 2(j+1), j < dims.          */
/* The floor must not depend on the libm in use: the double result is only  */
/* trusted when it is at least 2^-16 away from an integer, otherwise the    */
/* value is recomputed in long double and trusted at 2^-24; if even that is */
/* too close the function reports failure instead of guessing.              */
/* Returns 0 on success, -1 for invalid input, -2 if undecidable.           */
/* ------------------------------------------------------------------------ */
int orc_thresholds(int dims, double beta, uint32_t thr[3])
{
    if (dims != 2 && dims != 3) return -1;
    if (!(beta > 0.0)) return -1; /* rejects 0, negatives and NaN */
    for (int j = 0; j < 3; ++j) thr[j] = 0;
    for (int j = 0; j < dims; ++j) {
        int k = 2 * (j + 1);
        double x = 2.0 * beta * (double)k; /* exponent magnitude, > 0 */
        /* tiny x: 2^32 (1 - x) <= v < 2^32, so floor(v) = 2^32 - 1 exactly */
        if (x * 4294967296.0 < 0.5) { thr[j] = 0xFFFFFFFFu; continue; }
        double v = ldexp(exp(-x), 32);
        if (v < 0.5) { thr[j] = 0; continue; } /* 0 < true value < 1 */
        double f = v - floor(v);
        if (f >= 0x1p-16 && f <= 1.0 - 0x1p-16) {
            thr[j] = (uint32_t)floor(v);
            continue;
        }
        long double xl = 2.0L * (long double)beta * (long double)k;
        long double vl = ldexpl(expl(-xl), 32);
        long double fl = vl - floorl(vl);
        if (fl < 0x1p-24L || fl > 1.0L - 0x1p-24L) return -2;
        thr[j] = (uint32_t)floorl(vl);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Heat-bath thresholds (the alternative acceptance rule: each visited spin */
/* takes its conditional Boltzmann distribution given its neighbours, so    */
/* it flips with probability 1 / (1 + exp(beta dE)) = 1/(1 + exp(2 beta k))). */
/* Indexed by the number d = 0..2*dims of disagreeing neighbours, with      */
/* k = 2(dims - d): thb[d] = floor(2^32 / (1 + exp(4 beta (dims - d)))).     */
/* thb[dims] = 2^31 exactly.  Same exact-floor safeguards as above.         */
/* ------------------------------------------------------------------------ */
/* Two exact forms of the same number are used, each where it keeps full    */
/* relative precision: with x = 4 beta |dims - d| > 0,                      */
/*   2^32 / (1 + e^{+-x}) = 2^31 -+ delta,  delta = 2^31 tanh(x / 2),        */
/*   and for large x the small side 2^32 / (1 + e^x) directly.              */
static int heatbath_floor(int m, long double x, int wide, uint32_t *out)
{
    /* m > 0: floor(2^31 - delta); m < 0: floor(2^31 + delta)               */
    long double delta = wide ? ldexpl(tanhl(x / 2.0L), 31)
                             : (long double)ldexp(tanh((double)x / 2.0), 31);
    if (delta < 1073741824.0L) {           /* delta < 2^30: use delta      */
        if (delta < 1.0L) { *out = m > 0 ? 0x7FFFFFFFu : 0x80000000u; return 0; }
        long double f = delta - floorl(delta);
        if (f < (wide ? 0x1p-24L : 0x1p-16L) || f > 1.0L - (wide ? 0x1p-24L : 0x1p-16L))
            return 1;
        uint32_t fl = (uint32_t)floorl(delta);   /* delta not an integer    */
        *out = m > 0 ? 0x80000000u - fl - 1u : 0x80000000u + fl;
        return 0;
    }
    long double small = wide ? ldexpl(1.0L / (1.0L + expl(x)), 32)
                             : (long double)ldexp(1.0 / (1.0 + exp((double)x)), 32);
    if (small < 1.0L) { *out = m > 0 ? 0u : 0xFFFFFFFFu; return 0; }
    long double f = small - floorl(small);
    if (f < (wide ? 0x1p-24L : 0x1p-16L) || f > 1.0L - (wide ? 0x1p-24L : 0x1p-16L))
        return 1;
    uint32_t fl = (uint32_t)floorl(small);       /* small not an integer    */
    *out = m > 0 ? fl : 0xFFFFFFFFu - fl;        /* floor(2^32 - small)     */
    return 0;
}

int orc_thresholds_heatbath(int dims, double beta, uint32_t thb[7])
{
    if (dims != 2 && dims != 3) return -1;
    if (!(beta > 0.0)) return -1;
    for (int d = 0; d < 7; ++d) thb[d] = 0;
    for (int d = 0; d <= 2 * dims; ++d) {
        int m = dims - d; /* k / 2 */
        if (m == 0) { thb[d] = 0x80000000u; continue; }
        int am = m > 0 ? m : -m;
        if (isinf(beta) || 4.0 * beta * am > 800.0) {
            thb[d] = m > 0 ? 0u : 0xFFFFFFFFu;
            continue;
        }
        long double x = 4.0L * (long double)beta * (long double)am;
        if (heatbath_floor(m, x, 0, &thb[d]) == 0) continue;
        if (heatbath_floor(m, x, 1, &thb[d]) != 0) return -2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry                                                         */
/* ------------------------------------------------------------------------ */

static int64_t n_sites(int dims, int L)
{
    return dims == 2 ? (int64_t)L * L : (int64_t)L * L * L;
}

/* Sum of the 2*dims periodic neighbours of site (x,y,z); with L = 2 both
 * neighbours along an axis are the same site and it is counted twice. */
static int neighbour_sum(int dims, int L, const int8_t *s, int x, int y, int z)
{
    int64_t LL = (int64_t)L * L;
    int xp = (x + 1) % L, xm = (x + L - 1) % L;
    int yp = (y + 1) % L, ym = (y + L - 1) % L;
    int64_t base_z = (int64_t)z * LL;
    int h = s[base_z + (int64_t)y * L + xp] + s[base_z + (int64_t)y * L + xm] +
            s[base_z + (int64_t)yp * L + x] + s[base_z + (int64_t)ym * L + x];
    if (dims == 3) {
        int zp = (z + 1) % L, zm = (z + L - 1) % L;
        h += s[(int64_t)zp * LL + (int64_t)y * L + x] +
             s[(int64_t)zm * LL + (int64_t)y * L + x];
    }
    return h;
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. 2.2): forward bonds, so each lattice edge is counted  */
/* once for L >= 3 and an L = 2 pair once per direction (which is what the */
/* local update's dE = 2k assumes).                                         */
/* ------------------------------------------------------------------------ */

int64_t orc_energy(int dims, int L, const int8_t *s)
{
    int64_t e = 0;
    int zdim = dims == 3 ? L : 1;
    int64_t LL = (int64_t)L * L;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = (int64_t)z * LL + (int64_t)y * L + x;
                int sx = s[(int64_t)z * LL + (int64_t)y * L + (x + 1) % L];
                int sy = s[(int64_t)z * LL + (int64_t)((y + 1) % L) * L + x];
                int bond = sx + sy;
                if (dims == 3)
                    bond += s[(int64_t)((z + 1) % L) * LL + (int64_t)y * L + x];
                e -= (int64_t)s[i] * bond;
            }
    return e;
}

int64_t orc_magnetization(int dims, int L, const int8_t *s)
{
    int64_t m = 0, n = n_sites(dims, L);
    for (int64_t i = 0; i < n; ++i) m += s[i];
    return m;
}

/* ------------------------------------------------------------------------ */
/* Initial state (Sec. 2.2: spin up with probability p).                    */
/*   start 0 (hot):  p = 1/2, s_i = +1 iff u_i < 2^31 with                  */
/*                   u_i = Philox(seed; i>>2, 0, 0, TAG_INIT)[i & 3]        */
/*   start 1 (cold): all +1;  start 2: all -1.                              */
/* ------------------------------------------------------------------------ */
int orc_init(int dims, int L, uint64_t seed, int start, int8_t *s)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 1) return -1;
    int64_t n = n_sites(dims, L);
    for (int64_t i = 0; i < n; ++i) {
        if (start == 0) {
            uint32_t u = draw_word(seed, (uint32_t)(i >> 2), 0u, 0u, TAG_INIT,
                                   (unsigned)(i & 3));
            s[i] = u < 0x80000000u ? (int8_t)1 : (int8_t)-1;
        } else if (start == 1) {
            s[i] = 1;
        } else if (start == 2) {
            s[i] = -1;
        } else {
            return -1;
        }
    }
    return 0;
}

/* The Metropolis decision for one site (Sec. 2.2 steps 1-4), given the    */
/* local k = s_i * h_i (dE = 2k) and the draw that belongs to the site.     */
static int accept_flip(int k, const uint32_t thr[3], uint64_t seed,
                       uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       unsigned w)
{
    if (k <= 0) return 1;
    uint32_t u = draw_word(seed, c0, c1, c2, c3, w);
    return u < thr[k / 2 - 1];
}

/* The heat-bath decision: every visited site draws; it flips iff its draw  */
/* is below thb[d], d = (2*dims - k) / 2 the number of disagreeing          */
/* neighbours.                                                              */
static int heatbath_flip(int dims, int k, const uint32_t thb[7], uint64_t seed,
                         uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         unsigned w)
{
    int d = (2 * dims - k) / 2;
    uint32_t u = draw_word(seed, c0, c1, c2, c3, w);
    return u < thb[d];
}

/* ------------------------------------------------------------------------ */
/* One colour pass (Sec. 2.2: "a pass through all white or all black        */
/* sites").  Every site i of colour c is visited; it reads only sites of    */
/* the other colour, so the result does not depend on the visiting order.   */
/* Draw for site i in sweep t: Philox(seed; hh>>2, t, c, TAG_SWEEP)[hh & 3] */
/* with hh = i >> 1 (the site's index within its colour).  Requires L even. */
/* ------------------------------------------------------------------------ */
/* The decision for one site i = (x, y, z) of colour c in sweep t, reading */
/* its own spin and its neighbours from s: returns 1 iff the spin flips.    */
static int site_flips(int dims, int L, const int8_t *s, uint64_t seed,
                      const uint32_t *thr, uint32_t t, int c, int rule,
                      int x, int y, int z)
{
    int64_t i = (int64_t)z * L * L + (int64_t)y * L + x;
    int h = neighbour_sum(dims, L, s, x, y, z);
    int k = s[i] * h;
    int64_t hh = i >> 1;
    return rule == 0
        ? accept_flip(k, thr, seed, (uint32_t)(hh >> 2), t, (uint32_t)c,
                      TAG_SWEEP, (unsigned)(hh & 3))
        : heatbath_flip(dims, k, thr, seed, (uint32_t)(hh >> 2), t,
                        (uint32_t)c, TAG_SWEEP, (unsigned)(hh & 3));
}

int orc_half_sweep_rule(int dims, int L, int8_t *s, uint64_t seed,
                        const uint32_t *thr, uint32_t t, int c, int rule)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2 || (L & 1)) return -1;
    if (c != 0 && c != 1) return -1;
    int zdim = dims == 3 ? L : 1;
    int64_t LL = (int64_t)L * L;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != c) continue;
                int64_t i = (int64_t)z * LL + (int64_t)y * L + x;
                if (site_flips(dims, L, s, seed, thr, t, c, rule, x, y, z))
                    s[i] = (int8_t)-s[i];
            }
    return 0;
}

/* The spin that site i (canonical index) holds after its colour's pass of  */
/* sweep t, given the state s that pass starts from (for a white site: the  */
/* black sites already updated).  The same decision as the colour pass, for */
/* checking a large lattice one sampled site at a time.                     */
int orc_site_update(int dims, int L, const int8_t *s, uint64_t seed,
                    const uint32_t *thr, uint32_t t, int64_t i, int rule)
{
    if (dims != 2 && dims != 3) return 0;
    if (L < 2 || (L & 1)) return 0;
    int64_t n = dims == 3 ? (int64_t)L * L * L : (int64_t)L * L;
    if (i < 0 || i >= n) return 0;
    int x = (int)(i % L), y = (int)((i / L) % L), z = dims == 3 ? (int)(i / ((int64_t)L * L)) : 0;
    int c = (x + y + z) & 1;
    int f = site_flips(dims, L, s, seed, thr, t, c, rule, x, y, z);
    return f ? -s[i] : s[i];
}

/* Multi-hit Metropolis (a variant of Sec. 2.2's rule): each visited site   */
/* takes `hits` successive Metropolis trials, its neighbours fixed, the     */
/* spin it holds after a trial being the one the next trial may flip.       */
/* Trial m draws word hh & 3 of Philox(seed; hh >> 2, t, c + 2m, TAG_SWEEP); */
/* one hit is exactly the Metropolis pass.                                  */
int orc_half_sweep_multihit(int dims, int L, int8_t *s, uint64_t seed,
                            const uint32_t thr[3], uint32_t t, int c, int hits)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2 || (L & 1) || (c != 0 && c != 1) || hits < 1 || hits > 64) return -1;
    int zdim = dims == 3 ? L : 1;
    int64_t LL = (int64_t)L * L;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != c) continue;
                int64_t i = (int64_t)z * LL + (int64_t)y * L + x;
                int h = neighbour_sum(dims, L, s, x, y, z);
                int64_t hh = i >> 1;
                int sigma = s[i];
                for (int m = 0; m < hits; ++m)
                    if (accept_flip(sigma * h, thr, seed, (uint32_t)(hh >> 2), t,
                                    (uint32_t)(c + 2 * m), TAG_SWEEP, (unsigned)(hh & 3)))
                        sigma = -sigma;
                s[i] = (int8_t)sigma;
            }
    return 0;
}

int64_t orc_run_multihit(int dims, int L, double beta, uint64_t seed, int8_t *s,
                         uint32_t t0, int64_t nsweeps, int measure_every, int hits,
                         int64_t *E, int64_t *M, int64_t cap)
{
    uint32_t thr[3];
    int rc = orc_thresholds(dims, beta, thr);
    if (rc) return rc;
    if (measure_every < 1 || nsweeps < 0) return -1;
    int64_t nrec = 0;
    for (int64_t n = 0; n < nsweeps; ++n) {
        uint32_t t = t0 + (uint32_t)n;
        rc = orc_half_sweep_multihit(dims, L, s, seed, thr, t, 0, hits);
        if (rc == 0) rc = orc_half_sweep_multihit(dims, L, s, seed, thr, t, 1, hits);
        if (rc) return rc;
        if (((uint64_t)t + 1) % (uint64_t)measure_every == 0) {
            if (nrec < cap) {
                E[nrec] = orc_energy(dims, L, s);
                M[nrec] = orc_magnetization(dims, L, s);
            }
            ++nrec;
        }
    }
    return nrec;
}

/* Metropolis colour pass (rule 0). */
int orc_half_sweep(int dims, int L, int8_t *s, uint64_t seed,
                   const uint32_t thr[3], uint32_t t, int c)
{
    return orc_half_sweep_rule(dims, L, s, seed, thr, t, c, 0);
}

/* One sweep = black pass (colour 0) then white pass (colour 1). */
int orc_sweep_rule(int dims, int L, int8_t *s, uint64_t seed,
                   const uint32_t *thr, uint32_t t, int rule)
{
    int rc = orc_half_sweep_rule(dims, L, s, seed, thr, t, 0, rule);
    if (rc) return rc;
    return orc_half_sweep_rule(dims, L, s, seed, thr, t, 1, rule);
}

int orc_sweep(int dims, int L, int8_t *s, uint64_t seed,
              const uint32_t thr[3], uint32_t t)
{
    return orc_sweep_rule(dims, L, s, seed, thr, t, 0);
}

/* ------------------------------------------------------------------------ */
/* Sequential single-site Metropolis (the "standard" traversal Sec. 2.2     */
/* contrasts with the checkerboard), in canonical order i = 0..N-1.  Valid  */
/* for any L, including odd L where no checkerboard exists; it is used only */
/* to check the acceptance rule against exact enumeration on odd lattices.  */
/* Draw: Philox(seed; i>>2, t, 0, TAG_SEQUENTIAL)[i & 3].                   */
/* ------------------------------------------------------------------------ */
int orc_sweep_sequential(int dims, int L, int8_t *s, uint64_t seed,
                         const uint32_t thr[3], uint32_t t)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2) return -1;
    int zdim = dims == 3 ? L : 1;
    int64_t LL = (int64_t)L * L;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = (int64_t)z * LL + (int64_t)y * L + x;
                int k = s[i] * neighbour_sum(dims, L, s, x, y, z);
                if (accept_flip(k, thr, seed, (uint32_t)(i >> 2), t, 0u,
                                TAG_SEQUENTIAL, (unsigned)(i & 3)))
                    s[i] = (int8_t)-s[i];
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* A run: nsweeps sweeps numbered t0, t0+1, ...; after sweep t the energy   */
/* and magnetisation (recomputed from scratch) are recorded iff             */
/* (t + 1) % measure_every == 0.  Writes at most cap records and returns    */
/* their number (or a negative error).  mode 0 = checkerboard, 1 =          */
/* sequential, 2 = checkerboard heat bath.  The state s is updated in place. */
/* ------------------------------------------------------------------------ */
int64_t orc_run(int dims, int L, double beta, uint64_t seed, int8_t *s,
                uint32_t t0, int64_t nsweeps, int measure_every, int mode,
                int64_t *E, int64_t *M, int64_t cap)
{
    /* mode 0: checkerboard Metropolis; 1: sequential Metropolis;
       2: checkerboard heat bath */
    uint32_t thr[7];
    int rc = mode == 2 ? orc_thresholds_heatbath(dims, beta, thr)
                       : orc_thresholds(dims, beta, thr);
    if (rc) return rc;
    if (measure_every < 1 || nsweeps < 0) return -1;
    int64_t nrec = 0;
    for (int64_t n = 0; n < nsweeps; ++n) {
        uint32_t t = t0 + (uint32_t)n;
        rc = mode == 1 ? orc_sweep_sequential(dims, L, s, seed, thr, t)
                       : orc_sweep_rule(dims, L, s, seed, thr, t, mode == 2 ? 1 : 0);
        if (rc) return rc;
        if (((uint64_t)t + 1) % (uint64_t)measure_every == 0) {
            if (nrec < cap) {
                E[nrec] = orc_energy(dims, L, s);
                M[nrec] = orc_magnetization(dims, L, s);
            }
            ++nrec;
        }
    }
    return nrec;
}

/* ------------------------------------------------------------------------ */
/* Creutz's deterministic demon dynamics (Sec. 2.2 cites it: checkerboard   */
/* sweeps with a fully deterministic flip rule and no random numbers).      */
/* Readings (the paper gives no details):                                    */
/*   - every site carries a demon holding energy 4q, q = 0..qmax (the flip  */
/*     costs dE = 2k = 4 (dims - d) are multiples of 4);                     */
/*   - a site of the pass's colour flips iff its demon can pay or absorb    */
/*     the cost within its range, 0 <= q - (dims - d) <= qmax, and then     */
/*     q <- q - (dims - d); so E(S) + 4 sum q never changes;                */
/*   - after each sweep (black pass, white pass) every demon moves on by     */
/*     one half row within its colour: from the colour-c site in half row r */
/*     (r = y + L z) and half column xh = x >> 1 to the colour-c site in    */
/*     half row r + 1 (mod the number of half rows) and the same xh.        */
/* ------------------------------------------------------------------------ */
int orc_demon_half_sweep(int dims, int L, int8_t *s, uint8_t *q, int qmax, int c)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2 || (L & 1) || (c != 0 && c != 1)) return -1;
    if (qmax < 1 || qmax > 63) return -1;
    int zdim = dims == 3 ? L : 1;
    int64_t LL = (int64_t)L * L;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != c) continue;
                int64_t i = (int64_t)z * LL + (int64_t)y * L + x;
                int k = s[i] * neighbour_sum(dims, L, s, x, y, z); /* 2 (dims - d) */
                int qn = (int)q[i] - k / 2;
                if (qn >= 0 && qn <= qmax) {
                    s[i] = (int8_t)-s[i];
                    q[i] = (uint8_t)qn;
                }
            }
    return 0;
}

/* Move every demon one half row on (step = +1) or back (step = -1). */
int orc_demon_shift(int dims, int L, uint8_t *q, int step)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2 || (L & 1) || (step != 1 && step != -1)) return -1;
    int64_t n = n_sites(dims, L), LL = (int64_t)L * L;
    int64_t rows = dims == 3 ? LL : L;
    uint8_t *out = (uint8_t *)malloc((size_t)n);
    if (!out) return -2;
    int zdim = dims == 3 ? L : 1;
    for (int z = 0; z < zdim; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int c = (x + y + z) & 1;
                int64_t r = (int64_t)y + (int64_t)L * z;
                int64_t r2 = (r + step + rows) % rows;
                int y2 = (int)(r2 % L), z2 = dims == 3 ? (int)(r2 / L) : 0;
                int x2 = 2 * (x >> 1) + ((c + y2 + z2) & 1);
                out[(int64_t)z2 * LL + (int64_t)y2 * L + x2] =
                    q[(int64_t)z * LL + (int64_t)y * L + x];
            }
    memcpy(q, out, (size_t)n);
    free(out);
    return 0;
}

/* One demon sweep: black pass, white pass, demons move one half row on. */
int orc_demon_sweep(int dims, int L, int8_t *s, uint8_t *q, int qmax)
{
    int rc = orc_demon_half_sweep(dims, L, s, q, qmax, 0);
    if (rc == 0) rc = orc_demon_half_sweep(dims, L, s, q, qmax, 1);
    if (rc == 0) rc = orc_demon_shift(dims, L, q, 1);
    return rc;
}

/* nsweeps demon sweeps numbered t0, t0+1, ...; E and M recorded after sweep */
/* t iff (t + 1) % measure_every == 0.  Returns the number of records.      */
int64_t orc_demon_run(int dims, int L, int8_t *s, uint8_t *q, int qmax, uint32_t t0,
                      int64_t nsweeps, int measure_every, int64_t *E, int64_t *M,
                      int64_t cap)
{
    if (measure_every < 1 || nsweeps < 0) return -1;
    int64_t n = 0;
    for (int64_t k = 0; k < nsweeps; ++k) {
        int rc = orc_demon_sweep(dims, L, s, q, qmax);
        if (rc) return rc;
        uint64_t t = (uint64_t)t0 + (uint64_t)k;
        if ((t + 1) % (uint64_t)measure_every == 0) {
            if (n >= cap) return -3;
            E[n] = orc_energy(dims, L, s);
            M[n] = orc_magnetization(dims, L, s);
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Exact enumeration for Eq. 1: the number of states g(E, M) of a tiny      */
/* lattice, visiting all 2^N states in Gray-code order (one spin changes    */
/* per step, so E and M are updated by the local rule and re-checked from   */
/* scratch at the end).  hist has (2*dims*N + 1) * (2N + 1) int64 cells,    */
/* cell (E + dims*N) * (2N + 1) + (M + N).  N <= 30.                        */
/* ------------------------------------------------------------------------ */
int orc_enumerate(int dims, int L, int64_t *hist)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2) return -1;
    int64_t n = n_sites(dims, L);
    if (n > 30) return -1;
    int64_t ne = 2 * (int64_t)dims * n + 1, nm = 2 * n + 1;
    memset(hist, 0, (size_t)(ne * nm) * sizeof(int64_t));
    int8_t *s = (int8_t *)malloc((size_t)n);
    if (!s) return -3;
    for (int64_t i = 0; i < n; ++i) s[i] = -1;
    int64_t e = orc_energy(dims, L, s), m = orc_magnetization(dims, L, s);
    hist[(e + dims * n) * nm + (m + n)] += 1;
    uint64_t total = (uint64_t)1 << n;
    int64_t LL = (int64_t)L * L;
    for (uint64_t g = 1; g < total; ++g) {
        int j = 0;
        while (!((g >> j) & 1u)) ++j; /* position of the lowest set bit */
        int x = (int)(j % L), y = (int)((j / L) % L), z = (int)(j / LL);
        int h = neighbour_sum(dims, L, s, x, y, z);
        e += 2 * (int64_t)s[j] * h; /* dE of flipping s_j */
        m -= 2 * (int64_t)s[j];
        s[j] = (int8_t)-s[j];
        hist[(e + dims * n) * nm + (m + n)] += 1;
    }
    int ok = (e == orc_energy(dims, L, s)) && (m == orc_magnetization(dims, L, s));
    free(s);
    return ok ? 0 : -4;
}
