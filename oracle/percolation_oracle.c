/*
 * percolation_oracle.c -- plain, single-threaded CPU oracle for the site-
 * percolation model of Tomov et al. (2003), Sec. 2.3 (diffusion through a
 * porous medium).
 *
 * TEST INFRASTRUCTURE, like ising_oracle.c (built into the same library and
 * using its Philox4x32-10): only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the CUDA engine never calls it.
 *
 * What it follows (Sec. 2.3):
 *   - the porosity P is the probability that a site is a pore: every site
 *     draws R in [0, 1] and is a pore iff R <= P, solid otherwise;
 *   - an invasion point initialises the cluster, which then spreads through
 *     the pore space;
 *   - of interest: whether a spanning (percolating) cluster joins one end of
 *     the medium to the other, and the time to reach the steady state;
 *   - the porosity threshold for a spanning cluster in 2D is 0.592746
 *     (Sec. 5, results).
 *
 * Readings where the paper is silent:
 *   - 2D square lattices (the paper's) and 3D cubic ones, L^dims sites,
 *     canonical index i = x + L*y (+ L*L*z); open boundaries (a medium has
 *     ends); a site's neighbours are its 2*dims nearest sites inside the
 *     medium;
 *   - R = u / 2^32 with u = Philox(seed; i >> 2, 0, 0, TAG_PORE)[i & 3]
 *     (TAG_PORE = 3), so R <= P iff u <= floor(P * 2^32), the threshold
 *     capped at 2^32 - 1 (P = 1: every site is a pore);
 *   - spreading is a sequence of synchronous growth passes: in a pass a
 *     pore site joins the cluster iff one of its neighbours was in the
 *     cluster before the pass; the steady state is the first pass that adds
 *     nothing, and "steps" counts the passes that added sites (the largest
 *     growth distance from the invasion sites);
 *   - invasion sources: one site (POINT; an empty cluster if it is solid) or
 *     every pore of the first face (FACE), the sites whose slowest
 *     coordinate (y in 2D, z in 3D) is 0;
 *   - the cluster spans iff it holds a site of the first face and a site of
 *     the last face (slowest coordinate L - 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { TAG_PORE = 3 };
enum { PERC_POINT = 0, PERC_FACE = 1 };

/* floor(P * 2^32) capped at 2^32 - 1, for 0 <= P <= 1 (P * 2^32 is exact). */
int orc_perc_threshold(double P, uint32_t *thr)
{
    if (!(P >= 0.0 && P <= 1.0)) return -1;
    double v = floor(ldexp(P, 32));
    *thr = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
    return 0;
}

static int64_t perc_sites(int dims, int L)
{
    return dims == 3 ? (int64_t)L * L * L : (int64_t)L * L;
}

/* pore[i] = 1 iff u_i <= thr. */
int orc_perc_pores(int dims, int L, uint64_t seed, uint32_t thr, uint8_t *pore)
{
    if ((dims != 2 && dims != 3) || L < 1) return -1;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t n = perc_sites(dims, L);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)(i >> 2), 0u, 0u, TAG_PORE}, out[4];
        orc_philox4x32_10(ctr, key, out);
        pore[i] = out[i & 3] <= thr ? 1 : 0;
    }
    return 0;
}

/* Invade from the source and run growth passes to the steady state.  The   */
/* passes are taken one distance at a time: `front` holds the sites that    */
/* joined in the last pass, and the next pass adds every pore neighbour of  */
/* them not yet in the cluster (the same set as a pass over the whole       */
/* lattice, since a site can only join next to one that joined last).       */
int orc_perc_invade(int dims, int L, const uint8_t *pore, int source, int64_t site,
                    uint8_t *cluster, int64_t *size, int *spans, int64_t *steps)
{
    if ((dims != 2 && dims != 3) || L < 1) return -1;
    if (source != PERC_POINT && source != PERC_FACE) return -1;
    int64_t n = perc_sites(dims, L);
    if (source == PERC_POINT && (site < 0 || site >= n)) return -1;
    int64_t face = dims == 3 ? (int64_t)L * L : (int64_t)L; /* sites per face */
    int64_t *front = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!front || !next) {
        free(front);
        free(next);
        return -2;
    }
    memset(cluster, 0, (size_t)n);
    int64_t nf = 0, total = 0;
    if (source == PERC_POINT) {
        if (pore[site]) front[nf++] = site;
    } else {
        for (int64_t i = 0; i < face; ++i)
            if (pore[i]) front[nf++] = i;
    }
    for (int64_t k = 0; k < nf; ++k) cluster[front[k]] = 1;
    total = nf;
    int64_t passes = 0;
    int64_t LL = (int64_t)L * L;
    while (nf > 0) {
        int64_t nn = 0;
        for (int64_t k = 0; k < nf; ++k) {
            int64_t i = front[k];
            int64_t x = i % L, y = (i / L) % L, z = dims == 3 ? i / LL : 0;
            int64_t nb[6];
            int m = 0;
            if (x > 0) nb[m++] = i - 1;
            if (x < L - 1) nb[m++] = i + 1;
            if (y > 0) nb[m++] = i - L;
            if (y < L - 1) nb[m++] = i + L;
            if (dims == 3) {
                if (z > 0) nb[m++] = i - LL;
                if (z < L - 1) nb[m++] = i + LL;
            }
            for (int j = 0; j < m; ++j) {
                if (pore[nb[j]] && !cluster[nb[j]]) {
                    cluster[nb[j]] = 1;
                    next[nn++] = nb[j];
                }
            }
        }
        if (nn > 0) ++passes;
        total += nn;
        int64_t *tmp = front;
        front = next;
        next = tmp;
        nf = nn;
    }
    int first = 0, last = 0;
    for (int64_t i = 0; i < face; ++i) {
        if (cluster[i]) first = 1;
        if (cluster[n - face + i]) last = 1;
    }
    *size = total;
    *spans = first && last;
    *steps = passes;
    free(front);
    free(next);
    return 0;
}
