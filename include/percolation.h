/*
 * percolation.h -- C ABI of the GB300 site-percolation engine (the second
 * model of Tomov et al. (2003), Sec. 2.3: diffusion through a porous medium).
 *
 * A medium is a 2D square or 3D cubic lattice of L^dims sites with open
 * boundaries (it has two ends).  Sec. 2.3: every site draws R in [0, 1] and is
 * a pore iff R <= P (the porosity), solid otherwise; an invasion point starts
 * a cluster, which then spreads through the pore space; of interest are a
 * spanning cluster (one end to the other) and the time to the steady state.
 * The paper's porosity threshold for spanning in 2D is 0.592746 (Sec. 5).
 *
 * Here:
 *   - R = u / 2^32, u = word (i & 3) of Philox4x32-10(key = seed;
 *     counter = (i >> 2, 0, 0, 3)) for canonical site i = x + L*y (+ L*L*z),
 *     so a site is a pore iff u <= floor(P * 2^32) (capped at 2^32 - 1);
 *   - spreading is a sequence of synchronous growth passes: in a pass a pore
 *     site joins iff one of its 2*dims nearest neighbours inside the medium
 *     was in the cluster before the pass; the steady state is the first pass
 *     that adds nothing; `steps` counts the passes that added sites;
 *   - sources: PERC_POINT (one site; an empty cluster if it is solid) or
 *     PERC_FACE (every pore of the first face: slowest coordinate, y in 2D
 *     and z in 3D, equal to 0);
 *   - the cluster spans iff it holds a site of the first face and one of the
 *     last face (slowest coordinate L - 1).
 * Every result is a pure function of (dims, L, seed, P, source, site).
 *
 * Conventions as in ising.h: every call returns PERC_OK (0) or a negative
 * ISING_E* status code (same values); nothing aborts; a handle is used by one
 * thread at a time; work goes on the handle's stream; calls returning host
 * data synchronise it; the library owns the device memory of its handles.
 */
#ifndef PERCOLATION_GB300_H
#define PERCOLATION_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct perc_medium perc_medium; /* opaque, owned by the library */

enum { PERC_POINT = 0, PERC_FACE = 1 };

typedef struct perc_result {
    int64_t size;   /* sites in the cluster at the steady state */
    int32_t spans;  /* 1 iff the cluster joins the first and the last face */
    int32_t reserved;
    int64_t steps;  /* growth passes that added sites */
} perc_result;

/* Create a medium of L^dims sites (dims 2 or 3, L >= 1, L^dims <= 2^32) whose
 * draws use `seed`; every site starts solid.  Device memory: four bitmaps
 * (pores, cluster, two growth fronts) of L^(dims-1) rows of ceil(L/32)
 * words each.  Sets *out (NULL on failure). */
int perc_create(perc_medium **out, int dims, int L, uint64_t seed);

/* Draw the porosity field for porosity 0 <= P <= 1 (else ISING_EINVAL) on the
 * device; clears any cluster.  Asynchronous. */
int perc_generate(perc_medium *m, double porosity);

/* Invade from `source` (PERC_POINT with canonical `site`, or PERC_FACE; site
 * is ignored) and run growth passes until one adds nothing; fills *out.
 * Synchronises the stream (the host checks the pass counts in chunks). */
int perc_invade(perc_medium *m, int source, int64_t site, perc_result *out);

/* The porosity field / the cluster as L^dims uint8 0/1 values in canonical
 * order (host memory).  Synchronise. */
int perc_get_pores(perc_medium *m, uint8_t *host_out);
int perc_get_cluster(perc_medium *m, uint8_t *host_out);

/* How perc_invade runs its passes (same results either way):
 *   PERC_PASSES_AUTO (default): PERC_PASSES_GRAPH (measured the faster);
 *   PERC_PASSES_GRAPH: a CUDA graph of 64 chained pass launches (each placed
 *       on the SMs while the previous one drains) replayed until a pass adds
 *       nothing;
 *   PERC_PASSES_PERSISTENT: one cooperative launch (two CTAs per SM), the
 *       passes separated by a grid barrier whose every wait is bounded (about
 *       a second); a wait that runs out makes perc_invade return
 *       ISING_ETIMEOUT.
 * ISING_EINVAL for another value, or PERSISTENT where it cannot launch. */
enum { PERC_PASSES_AUTO = 0, PERC_PASSES_GRAPH = 1, PERC_PASSES_PERSISTENT = 2 };
int perc_set_passes(perc_medium *m, int mode);

/* Use this CUDA stream (a cudaStream_t, may be NULL) for later work. */
int perc_set_stream(perc_medium *m, void *stream);

/* Free the medium.  NULL is accepted. */
void perc_destroy(perc_medium *m);

/*
 * Many independent media in one launch (for spanning probabilities): medium k
 * uses seeds[k]; all share dims, L, P, source and site.  One CTA per medium
 * holds its pores, cluster and fronts in shared memory, so L is limited to
 * 2D L <= 512 and 3D L <= 64 (ISING_EINVAL beyond).  results: n host structs.
 * clusters_dev: NULL, or caller-owned DEVICE memory of n * L^dims bytes that
 * receives each cluster (0/1, canonical order).  Synchronises `stream`.
 */
int perc_batch(int dims, int L, double porosity, const uint64_t *seeds, int n, int source,
               int64_t site, perc_result *results, uint8_t *clusters_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PERCOLATION_GB300_H */
