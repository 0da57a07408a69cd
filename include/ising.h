/*
 * ising.h -- C ABI of the GB300 checkerboard-Metropolis Ising engine.
 *
 * The engine simulates the Ising model of Tomov et al. (2003), Sec. 2.2: spins
 * s = +-1 on a periodic 2D square or 3D cubic lattice of linear size L, energy
 * E = -sum over nearest-neighbour bonds of s_j s_k (J = 1, no field) and
 * magnetisation M = sum of s.  One sweep is a pass over all black sites
 * (x+y[+z] even) followed by a pass over all white sites (Sec. 2.2,
 * "consecutive black and white sweeps"); each site flips by the Metropolis
 * rule of Sec. 2.2 with dE = 2k, k = s_i * (sum of its neighbours): k <= 0
 * always flips, k > 0 flips iff u < floor(exp(-2 beta k) 2^32), where u is the
 * 32-bit Philox4x32-10 draw keyed by (seed) and counted by (site, sweep,
 * colour), so results do not depend on layout or launch shape.  The per-sweep
 * E and M are reduced inside the sweep kernels.
 *
 * Conventions shared by every call:
 *   - Canonical site order: i = x + L*y (+ L*L*z), x fastest; spins are int8
 *     +1 / -1 in host and device spin buffers.
 *   - Every call returns ISING_OK (0) or a negative ISING_E* code; nothing
 *     aborts.  ising_strerror() names a code.  After ISING_ECUDA the handle
 *     should be destroyed.
 *   - Handles are not thread-safe: one handle, one thread at a time.
 *   - Work is issued on the handle's CUDA stream (default: the legacy default
 *     stream); calls that return host data synchronise that stream.
 *   - The library owns all device memory it allocates for a handle and frees
 *     it in ising_destroy().  Lattice memory (spins, demons, records) comes
 *     from a stream-ordered pool the library keeps per device: a destroyed
 *     lattice's blocks stay reserved for the next one (creating and
 *     destroying lattices never synchronises the device) until
 *     ising_release_cached_memory() hands them back.
 */
#ifndef ISING_GB300_H
#define ISING_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ising_lattice ising_lattice; /* opaque, owned by the library */

/* Spin layouts on the device. */
enum {
    ISING_INT8 = 0,    /* one int8 per site, one array per colour (the two-lattice
                          checkerboard of Sec. 5), row-major half rows */
    ISING_BITPACK = 1, /* 32 same-colour sites per uint32 word, each half row
                          padded to whole words */
    ISING_AUTO = 2     /* the engine picks (bit-packed); never changes results */
};

/* Kernels for the int8 colour pass (same results; see ising_set_kernel). */
enum {
    ISING_KERNEL_AUTO = 0,  /* a registered configuration (ising_set_int8_config), else staged
                               for 2D with 4096 <= L <= 16384 and strip otherwise (measured) */
    ISING_KERNEL_STRIP = 1, /* per-thread row strips, neighbour rows in registers */
    ISING_KERNEL_TMA = 2    /* tiles staged in shared memory by bulk (TMA) copies */
};

/*
 * Local update rules of a colour pass (see ising_set_rule).  Both visit the
 * same sites with the same draw u per site and keep the Boltzmann
 * distribution P(S) of Sec. 2.2 stationary.  With d the number of the site's
 * 2*dims neighbours that disagree with it (dE = 4 (dims - d)):
 *   METROPOLIS (Sec. 2.2, steps 1-4): d >= dims flips without a draw; otherwise
 *       flip iff u < floor(exp(-beta dE) 2^32).
 *   HEATBATH: the site takes its conditional Boltzmann distribution given its
 *       neighbours, P(S') / (P(S) + P(S')) = 1 / (1 + exp(beta dE)) for the
 *       flipped state: every site draws and flips iff
 *       u < floor(2^32 / (1 + exp(4 beta (dims - d)))).
 *   MULTIHIT: Metropolis with `hits` successive trials per visit, the
 *       neighbours fixed (each trial as above, on the spin the site then
 *       holds); trial m draws with counter word 2 = c + 2m instead of c, so
 *       one hit is exactly METROPOLIS.  Still samples P(S); fewer rejections.
 *   DEMON: Creutz's deterministic dynamics, which Sec. 2.2 cites (checkerboard
 *       sweeps, no random numbers).  Every site carries a demon of energy 4q,
 *       q = 0..qmax; a site flips iff 0 <= q - (dims - d) <= qmax, and its
 *       demon keeps q - (dims - d), so E + 4 sum q is conserved (the
 *       microcanonical ensemble; beta and the draws are not used).  After each
 *       sweep every demon moves on by one half row within its colour: from the
 *       colour-c site in half row r = y + L z, half column x >> 1, to the
 *       colour-c site in half row r + 1 (mod L^(dims-1)), same half column.
 */
enum {
    ISING_RULE_METROPOLIS = 0,
    ISING_RULE_HEATBATH = 1,
    ISING_RULE_DEMON = 2,    /* deterministic demon dynamics (ising_set_demons) */
    ISING_RULE_MULTIHIT = 3  /* Metropolis with several trials per visit (ising_set_hits) */
};

/* Initial states (Sec. 2.2: spins up with probability p). */
enum {
    ISING_HOT = 0,       /* p = 1/2: s_i = +1 iff Philox(seed; i>>2, 0, 0, 1)[i&3] < 2^31 */
    ISING_COLD_UP = 1,   /* p = 1: all +1 */
    ISING_COLD_DOWN = 2  /* p = 0: all -1 */
};

/* Status codes. */
enum {
    ISING_OK = 0,
    ISING_EINVAL = -1,   /* invalid argument */
    ISING_ENOMEM = -2,   /* device or host allocation failed */
    ISING_ECUDA = -3,    /* a CUDA call failed */
    ISING_ETIMEOUT = -4, /* a bounded device wait gave up */
    ISING_EBUDGET = -5,  /* would exceed a memory budget */
    ISING_ERANGE = -6    /* counter/capacity exhausted or buffer too small */
};

typedef struct ising_info_t {
    int dims;              /* 2 or 3 */
    int L;                 /* linear size */
    int layout;            /* ISING_INT8 or ISING_BITPACK (never AUTO) */
    int rule;              /* ISING_RULE_METROPOLIS or ISING_RULE_HEATBATH */
    double beta;           /* inverse temperature J/kT */
    uint64_t seed;         /* Philox key */
    uint64_t sweeps_done;  /* global sweep counter t (next sweep's index) */
    uint64_t sites;        /* L^dims */
    uint64_t device_bytes; /* device memory held by the spin arrays */
    int64_t pending_records; /* E/M records not yet read by ising_observables */
} ising_info_t;

/*
 * Create a lattice and put it in the hot start (ISING_HOT), sweep counter 0.
 *   out    receives the handle (set to NULL on failure).
 *   dims   2 or 3.
 *   L      even, >= 2 (odd L has no valid checkerboard on a torus: the wrap
 *          bond would join two sites of one colour); L^dims <= 2^32.
 *   beta   > 0 (may be +inf for a zero-temperature quench).  The thresholds
 *          of both rules (ISING_RULE_*) are built on the host; a beta for
 *          which one of them lies too close to an integer boundary to decide
 *          its floor at long-double precision is rejected with ISING_EINVAL.
 *   seed   64-bit Philox key (low word, high word).
 *   layout ISING_INT8, ISING_BITPACK or ISING_AUTO.
 * Allocates device memory; issues the init kernel on the default stream.
 */
int ising_create(ising_lattice **out, int dims, int L, double beta,
                 uint64_t seed, int layout);

/* Re-initialise the spins (ISING_HOT / ISING_COLD_UP / ISING_COLD_DOWN), reset
 * the sweep counter to 0 and drop pending E/M records. Asynchronous. */
int ising_init(ising_lattice *lat, int start);

/*
 * Run n >= 0 sweeps, numbered t, t+1, ..., t+n-1 (t = sweeps done so far).
 * After sweep number u the fused kernels record (E, M) iff
 * (u + 1) % measure_every == 0 (measure_every >= 1).  Asynchronous on the
 * handle's stream; may grow the device record buffer.  ISING_ERANGE if the
 * counter would pass 2^32 - 1.  The colour passes are launched with
 * programmatic stream serialisation: a pass may be scheduled while the kernel
 * before it in the stream drains, and touches no memory until that kernel has
 * completed, so stream order holds as for ordinary launches (an event or a
 * copy between two passes only keeps them from overlapping their launch).
 */
int ising_sweep(ising_lattice *lat, int64_t n, int measure_every);

/*
 * Read the pending E/M records (oldest first) and clear them.  Synchronises
 * the stream once (the records are copied through a pinned staging buffer
 * that the handle keeps).  *count receives the number pending.  With
 * E == NULL or M == NULL only the count is reported.  If cap < pending
 * nothing is copied, nothing is cleared and ISING_ERANGE is returned.  On
 * ISING_ETIMEOUT (a bounded wait gave up since the last check) the records of
 * this read are dropped.
 */
int ising_observables(ising_lattice *lat, int64_t *E, int64_t *M, int64_t cap,
                      int64_t *count);

/*
 * The same read without waiting: enqueue on the handle's stream a copy of the
 * pending records into `pairs` (host memory, pinned for an asynchronous copy:
 * cap pairs of int64 (E, M), oldest first) and clear them; *count receives
 * their number at once.  The values are in place once the stream has passed
 * this point (an event, ising_synchronize, or any call that syncs), so a
 * caller can read sweep k's records while sweep k+1 runs.  No timeout check
 * is made here (ising_synchronize makes it).  If cap < pending nothing is
 * copied or cleared and ISING_ERANGE is returned.
 */
int ising_observables_async(ising_lattice *lat, int64_t *pairs, int64_t cap, int64_t *count);

/*
 * The same asynchronous read for n lattices at once, with one queued kernel
 * instead of a copy and a clear per lattice (the per-sweep records of Sec. 2.2
 * for a whole set of lattices).  All n lattices must use the same stream; the
 * work goes there.  counts[i] (host, n entries) receives lattice i's number of
 * pending records at once, and its records go to pairs[2 * off_i ...] (int64
 * (E, M) pairs, oldest first) with off_i = counts[0] + ... + counts[i - 1];
 * they are cleared on the device (a handle listed twice gets them at its first
 * entry and a count of 0 at the second).  `pairs` must be pinned host memory the
 * device can write (cudaHostAlloc, cudaMallocHost or cudaHostRegister, as
 * torch's pin_memory is); the kernel stores into it directly.  The values are
 * in place once the stream has passed this point.  ISING_EINVAL for n < 1, a
 * NULL argument or lattice, lattices on different streams, or `pairs` not
 * device-writable (nothing is queued or cleared then); ISING_ERANGE if cap
 * (pairs) is below the total pending, likewise with nothing queued.
 */
int ising_observables_gather(ising_lattice *const *lats, int n, int64_t *pairs, int64_t cap,
                             int64_t *counts);

/*
 * ising_observables_gather, and then the device stores `value` into *flag
 * (pinned host memory, as for `pairs`) after the records are in place and
 * visible to the host: a host that reads `value` there may read the records
 * without an event or a synchronisation (the flag is written even when no
 * record is pending).  ISING_EINVAL also for a flag that is not
 * device-writable host memory.
 */
int ising_observables_gather_signal(ising_lattice *const *lats, int n, int64_t *pairs,
                                    int64_t cap, int64_t *counts, int64_t *flag, int64_t value);

/* Copy the spins to host memory in canonical order (L^dims int8).  Syncs.
 * Pinned host memory is written by the export kernel directly; pageable
 * memory goes through a device buffer taken for the call.  ISING_EINVAL if
 * an ising_set_spins_async of this handle met an invalid value (see there). */
int ising_get_spins(ising_lattice *lat, int8_t *host_out);

/* Load spins (canonical int8 +-1, host memory) and set the sweep counter to
 * t; pending records are dropped.  Values other than +-1 give ISING_EINVAL
 * (checked on the host before anything changes).  Syncs.  Pinned host memory
 * is read by the import kernel directly, pageable memory through a device
 * buffer taken for the call. */
int ising_set_spins(ising_lattice *lat, const int8_t *host_in, uint64_t t);

/*
 * ising_set_spins without waiting (checkpoint resume, or the initial state
 * of a job, overlapped with other work).  `in` holds L^dims canonical int8
 * spins in memory the device can read directly: device memory, or pinned
 * host memory (cudaHostAlloc, cudaMallocHost, cudaHostRegister, as torch's
 * pin_memory is), which the import kernel reads over the host link with no
 * staging copy.  Sets the sweep counter to t and drops pending records, then
 * returns; the kernel runs in the handle's stream order, so `in` must stay
 * unchanged until the stream has passed this point.  The values are checked
 * on the device: if a byte is neither +1 nor -1, the next ising_synchronize,
 * ising_observables or ising_get_spins of this handle returns ISING_EINVAL
 * (once), and the spins are undefined until the next ising_init or
 * ising_set_spins.  ISING_EINVAL at once for memory the device cannot read
 * (pageable host memory: use ising_set_spins); ISING_ERANGE for
 * t > 2^32.
 */
int ising_set_spins_async(ising_lattice *lat, const int8_t *in, uint64_t t);

/* Write the spins in canonical order (L^dims int8) into memory the device can
 * write directly -- device memory or pinned host memory -- without waiting:
 * the export kernel runs in the handle's stream order and the values are in
 * place once the stream has passed this point (an event, ising_synchronize).
 * ISING_EINVAL for memory the device cannot write. */
int ising_get_spins_async(ising_lattice *lat, int8_t *out);

/* Write the spins in canonical order into caller-owned DEVICE memory
 * (L^dims bytes).  Asynchronous on the handle's stream. */
int ising_export_device(ising_lattice *lat, int8_t *dev_out);

/* Choose the int8 pass kernel of a lattice (ISING_KERNEL_*).  The staged
 * kernel needs L % 32 == 0 and tiles that fit in shared memory; otherwise, and
 * for the bit-packed layout, the choice is recorded but the general kernels
 * run.  Results never depend on it. */
int ising_set_kernel(ising_lattice *lat, int kernel);

/* The int8 pass kernel the lattice's sweeps run, with ISING_KERNEL_AUTO and the
 * size limits resolved: ISING_KERNEL_TMA or ISING_KERNEL_STRIP (which also
 * stands for the general kernel used when L/2 is not a multiple of 16).  For
 * the bit-packed layout *kernel is set to -1. */
int ising_get_kernel(const ising_lattice *lat, int *kernel);

/*
 * Tuned int8 pass configurations (for the autotuner).  A configuration names
 * the kernel of the int8 colour pass and, for the staged kernel, its shape:
 *   kernel       ISING_KERNEL_STRIP or ISING_KERNEL_TMA;
 *   tile_rows    half rows per staged tile (of one plane in 3D): 1 (each
 *                thread one row at a time) or 2, 4, ..., 64 (each thread two
 *                rows at a time); 0: the engine's default for L (about 8 KiB
 *                of own-colour rows);
 *   ctas_per_sm  resident CTAs per SM of the staged kernel, 1..8 (fewer if
 *                they do not fit); 0: as many as fit.
 * Results never depend on the configuration.
 */
typedef struct ising_int8_config {
    int kernel;
    int tile_rows;
    int ctas_per_sm;
} ising_int8_config;

/* Register `cfg` for int8 lattices of `dims` with L_min <= L <= L_max: their
 * ISING_KERNEL_AUTO passes (and, for tile_rows and ctas_per_sm, their
 * ISING_KERNEL_TMA passes) run it from the next sweep on; a later
 * registration overrides an earlier one where they overlap; a configuration
 * the staged kernel cannot take for some L (tile rows not dividing L, stages
 * too large for shared memory) runs the general kernels there.  Process-wide
 * (all devices); thread-safe.  ISING_EINVAL for dims not in {2, 3}, an empty
 * range or a value out of range. */
int ising_set_int8_config(int dims, int L_min, int L_max, const ising_int8_config *cfg);

/* Drop every registered configuration (ISING_KERNEL_AUTO returns to the
 * built-in choice: the staged kernel for 2D 4096 <= L <= 16384). */
int ising_clear_int8_configs(void);

/* The configuration the lattice's int8 passes run now (registered or
 * built-in, size limits resolved); kernel = -1 for the bit-packed layout. */
int ising_get_int8_config(const ising_lattice *lat, ising_int8_config *out);

/* The engine's counter-based generator on the device: for c0 = 0..n-1,
 * dev_out[4*c0 + j] = word j of Philox4x32-10(key = seed; counter =
 * (c0, c1, c2, c3)) (Salmon et al., SC'11), the same function every kernel
 * draws from.  dev_out: caller-owned device memory of 4n uint32.  Asynchronous
 * on `stream`.  For checking the generator and measuring its throughput. */
int ising_philox_fill(uint32_t *dev_out, uint32_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint64_t seed, void *stream);

/* Throughput probe of the same generator: blocks x threads threads (threads
 * 128 or 256) each run iters x chains calls, counter word 0 = gid * iters *
 * chains + k (distinct for every call), word 1 = 5, words 2 and 3 = 0 (the
 * uniform words of a sweep's draws), and fold the four words of every call
 * into one uint32 by xor, stored at dev_out[gid] (caller-owned device memory,
 * blocks x threads words).  variant 0 is the form every kernel uses (one
 * widening 32x32 -> 64-bit multiply per product), 1 the same function with
 * separate low and high 32-bit multiplies; chains (4 or 8) independent calls
 * per step.  Asynchronous on `stream`; calls/s = blocks x threads x iters x
 * chains / time.  ISING_EINVAL for other shapes, ISING_ERANGE if the
 * counters would pass 2^32.  For measuring the integer ceiling of a pass. */
int ising_philox_probe(uint32_t *dev_out, int blocks, int threads, uint32_t iters, int variant,
                       int chains, uint64_t seed, void *stream);

/* Test hook for the bounded waits: while `on` is nonzero, every staged (TMA)
 * pass expects more bytes on its first tile than are ever copied, so its wait
 * runs out after about a second, the kernel returns early and the next
 * ising_synchronize / ising_observables reports ISING_ETIMEOUT; and every
 * persistent percolation launch (perc_invade) has one CTA leave before the
 * first grid barrier, so the others' waits run out and perc_invade returns
 * ISING_ETIMEOUT.  The results of such a pass or invasion are not defined.
 * Off by default. */
int ising_test_inject_timeout(int on);

/* Use this CUDA stream (a cudaStream_t, may be NULL = legacy default stream)
 * for all later work of the handle.  The caller keeps ownership. */
int ising_set_stream(ising_lattice *lat, void *stream);

/* The thresholds in use: out[j] = floor(exp(-2 beta (2j+2)) 2^32) for
 * j < dims, 0 beyond. */
int ising_thresholds(const ising_lattice *lat, uint32_t out[3]);

/* The same thresholds for (dims, beta) without a handle or a GPU (host-only
 * computation; ISING_EINVAL for dims not in {2,3}, beta <= 0 or NaN, or a
 * beta whose floor cannot be decided as described at ising_create). */
int ising_compute_thresholds(int dims, double beta, uint32_t out[3]);

/* Select the local update rule (ISING_RULE_*) for the lattice's later
 * sweeps; the default is ISING_RULE_METROPOLIS.  Both thresholds tables are
 * built at ising_create; ISING_RULE_DEMON needs demons (ising_set_demons)
 * first.  ISING_EINVAL for an invalid handle or rule.  The sweep counter and
 * records are unchanged. */
int ising_set_rule(ising_lattice *lat, int rule);

/* Trials per visit of ISING_RULE_MULTIHIT, 1 <= hits <= 64 (default 2;
 * ISING_EINVAL otherwise).  The rule itself is chosen by ising_set_rule. */
int ising_set_hits(ising_lattice *lat, int hits);

/* Load the demons of ISING_RULE_DEMON.  host_q: L^dims bytes in canonical
 * order, each <= qmax; or NULL, every demon = fill (0 <= fill <= qmax).
 * int8 layout: 1 <= qmax <= 63, one byte per site.  Bit-packed layout:
 * qmax must be 3 (two demon bit planes; ISING_EINVAL otherwise).  The first
 * call allocates the demon arrays (the size of the spin arrays, twice that
 * when packed).  Syncs.  The spins, the sweep counter and the rule are
 * unchanged. */
int ising_set_demons(ising_lattice *lat, const uint8_t *host_q, int fill, int qmax);

/* The demons in canonical order (L^dims bytes of host memory), as the next
 * sweep will see them; ISING_EINVAL if none were loaded.  Syncs. */
int ising_get_demons(ising_lattice *lat, uint8_t *host_out);

/* The heat-bath thresholds for (dims, beta) without a handle or a GPU:
 * out[d] = floor(2^32 / (1 + exp(4 beta (dims - d)))) for d = 0..2*dims
 * (out[dims] = 2^31), 0 beyond; out has 7 entries.  Errors as at
 * ising_compute_thresholds. */
int ising_compute_thresholds_heatbath(int dims, double beta, uint32_t out[7]);

/* Describe the handle. */
int ising_get_info(const ising_lattice *lat, ising_info_t *out);

/* Block until the handle's stream is idle; ISING_ETIMEOUT if a kernel gave up
 * on a bounded wait since the last check (the flag is then cleared). */
int ising_synchronize(ising_lattice *lat);

/* Free everything the handle owns.  NULL is accepted.  Does not wait for the
 * handle's queued work: its device memory returns to the library's pool in
 * the handle's stream order (the stream must still exist); only a handle
 * that holds pinned host buffers (after ising_observables or
 * ising_set_spins_async) waits for its stream first. */
void ising_destroy(ising_lattice *lat);

/* Return the memory the library's pool on the current device keeps for
 * reuse (blocks of destroyed lattices) to the system.  Synchronises the
 * device first. */
int ising_release_cached_memory(void);

/*
 * Batched form: many independent lattices (any mix of dims, L, layout, beta,
 * seed) advanced by one persistent launch, with the same arithmetic and draws
 * as ising_sweep, so each lattice ends bit-identical to running it alone.
 * Lattices with at least huge_sites sites are advanced by the per-lattice
 * pass kernels (each pass over the whole GPU) on the batch stream; the others
 * are jobs of one persistent kernel, taken largest first from a device work
 * queue: lattices with at least big_sites sites are run by a thread-block
 * cluster of cluster_size CTAs (colour passes separated by the hardware
 * cluster barrier), smaller ones by a single CTA each.  The launch is captured once
 * in a CUDA graph and replayed; each launch advances lattice i by sweeps[i]
 * sweeps and records E/M after sweep u iff (u + 1) % measure_every[i] == 0.
 */
typedef struct ising_batch ising_batch; /* opaque */

typedef struct ising_batch_opts {
    int block_threads;  /* threads per CTA: 128 or 256 (0: 256) */
    int cluster_size;   /* CTAs per cluster for large lattices, 1..8 (0: 4);
                           1 runs every lattice on a single CTA */
    int64_t big_sites;  /* size threshold of the cluster queue (0: 2^18) */
    int use_graph;      /* >= 0: capture the persistent launch in a CUDA graph and
                           replay it; < 0: plain launches */
    int64_t huge_sites; /* lattices this large use the per-lattice kernels
                           (0: 2^22; < 0: never) */
} ising_batch_opts;

/*
 * Build a batch over n distinct lattices of the current device.  sweeps[i] >= 0
 * sweeps per launch for lattice i; measure_every may be NULL (every sweep) or
 * give a value >= 1 per lattice; opts may be NULL.  All lattices are moved to
 * `stream` (as by ising_set_stream).  The batch borrows the handles: between
 * ising_batch_launch and ising_batch_sync they must not be used directly, and
 * they must outlive the batch.  Device memory: a job table (96 B per lattice).
 * Lattices of each update rule (ISING_RULE_*) form their own queues, run by
 * one persistent launch per rule present; demon-dynamics and multi-hit
 * lattices are advanced by the per-lattice kernels like the huge ones.  A lattice's rule
 * must not change while the batch exists (ising_batch_launch then returns
 * ISING_EINVAL).
 */
int ising_batch_create(ising_batch **out, ising_lattice *const *lats, int n,
                       const int64_t *sweeps, const int *measure_every,
                       const ising_batch_opts *opts, void *stream);

/* Replace the batch's lattices, sweep counts and measurement intervals (the
 * same rules as at ising_batch_create; the options stay) for its next launch,
 * reusing its device tables (they grow, in stream order, when n exceeds every
 * earlier size).  May be called while an earlier launch of the batch is still
 * running: that launch keeps its own lattices and counts, and the new ones
 * follow it on the batch stream.  The new lattices are moved to the batch
 * stream; a captured graph is dropped and recaptured at the next launch.
 * For loops that change the set every round (continuous batching) without
 * creating and destroying a batch each time. */
int ising_batch_update(ising_batch *b, ising_lattice *const *lats, int n,
                       const int64_t *sweeps, const int *measure_every);

/* Advance every lattice of the batch by its sweeps (asynchronous). */
int ising_batch_launch(ising_batch *b);

/* Wait for the batch's launches; afterwards the lattices may be used
 * directly (ising_observables, ising_get_spins, ...). */
int ising_batch_sync(ising_batch *b);

/* Resident grid size, the number of jobs in the cluster / CTA queues and the
 * number of lattices advanced by the per-lattice kernels. */
int ising_batch_info(const ising_batch *b, int *grid, int *n_big, int *n_small, int *n_huge);

/* Free the batch (not the lattices).  NULL is accepted. */
void ising_batch_destroy(ising_batch *b);

/*
 * The batched form in one call: advance lattice i of lats[0..n-1] by
 * sweeps[i] sweeps (Sec. 2.2's black and white passes, the same arithmetic and
 * draws as ising_sweep) in one persistent launch on `stream`, recording E/M
 * after sweep u iff (u + 1) % measure_every == 0 into each handle's own record
 * buffer (read them with ising_observables or ising_observables_gather).
 * Equivalent to ising_batch_create (default options, no graph) +
 * ising_batch_launch + ising_batch_sync + ising_batch_destroy: it moves the
 * lattices to `stream`, allocates the job table for the call, and returns
 * once the sweeps are done.  Errors as at those calls (ISING_EINVAL for
 * n < 1, measure_every < 1, a NULL or repeated lattice, a negative count).
 */
int ising_batch_run(ising_lattice *const *lats, int n, const int64_t *sweeps, int measure_every,
                    void *stream);

/*
 * ising_batch_run_static -- the batched launch for callers that cannot
 * allocate device memory while they run.  (An engine facility; the paper has
 * no counterpart.)  Some callers must not allocate once running: a real-time
 * or latency-bound loop where cudaMalloc would stall the device, code that
 * owns a fixed memory pool, or a host that has reserved all device memory for
 * its lattices up front.  This call advances lattice i by sweeps[i] sweeps in
 * one persistent launch on `stream`, like ising_batch_create + launch, but
 * allocates nothing: its work queue (job table, queue order, counters) lives
 * in one file-scope device array of fixed size, at most 2048 lattices per
 * call (more gives ISING_ERANGE before any work is issued); every GPU that
 * loads the library holds that array, about 200 KiB, until the process exits.
 *
 *   lats, n        n distinct lattices of the current device (1 <= n <= 2048),
 *                  each already on `stream` (ising_set_stream): the work is
 *                  ordered against the handles' own calls by that stream
 *                  alone, so a lattice on another stream gives ISING_EINVAL
 *                  (nothing issued).
 *   sweeps         n sweep counts (>= 0).
 *   measure_every  NULL (every sweep) or n intervals (>= 1): E/M is recorded
 *                  after sweep u iff (u + 1) % measure_every[i] == 0.
 *   records        caller-owned DEVICE buffer of (E, M) int64 pairs.  Lattice
 *                  i's records follow those of lattices 0..i-1, in sweep
 *                  order.  The call zeroes and fills only the pairs it
 *                  writes; records_cap is the number of pairs available and
 *                  must cover them all (else ISING_ERANGE, nothing issued).
 *                  The handles' own record buffers are not touched.
 *   opts           block_threads, cluster_size and big_sites as for
 *                  ising_batch_create (NULL: defaults); every lattice runs in
 *                  the persistent kernel (huge_sites and use_graph are ignored),
 *                  so ISING_RULE_DEMON and ISING_RULE_MULTIHIT lattices are
 *                  refused (ISING_EINVAL).
 * The spins and sweep counters of the handles advance as with ising_sweep.
 * The first call on a device looks up the array's device address and the
 * resident grid size; make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents, so
 * calls whose work overlaps on the GPU (e.g. issued on two streams without
 * ordering) race: order them on one stream or synchronise between them.
 */
int ising_batch_run_static(ising_lattice *const *lats, int n, const int64_t *sweeps,
                           const int *measure_every, int64_t *records, int64_t records_cap,
                           const ising_batch_opts *opts, void *stream);

/* Static description of a status code. */
const char *ising_strerror(int code);

/* Library version string. */
const char *ising_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISING_GB300_H */
