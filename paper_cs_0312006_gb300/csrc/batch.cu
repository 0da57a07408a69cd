// batch.cu -- many independent lattices of uneven size in one persistent
// launch (the batched form of the checkerboard sweep; same arithmetic, same
// draws, so each lattice's result is identical to running it alone).
//
// Lattices of at least huge_sites sites are advanced with the per-lattice
// pass kernels (each pass spread over the whole GPU), issued on the batch's
// stream ahead of the persistent launch; everything smaller goes through the
// persistent kernel.
//
// Work queue: one job per lattice, holding everything its sweeps need (spin
// arrays, thresholds, key, first sweep index, sweep count, measurement
// interval, record slots).  Jobs are ordered by work (sites x sweeps),
// largest first, and split in two queues at a size threshold:
//   - large jobs are run by a thread-block cluster: the CTAs of the cluster
//     share the job's words, and consecutive colour passes are separated by
//     the hardware cluster barrier (release/acquire at cluster scope), with
//     the other colour read through L2 so that words written by another CTA
//     of the cluster are seen;
//   - small jobs are run by one CTA each, passes separated by __syncthreads.
// Each cluster (then each CTA) takes the next job with one atomicAdd on a
// queue counter and runs all of the job's sweeps before taking another, so
// there is no inter-CTA waiting other than the cluster barrier.  At the end of
// a job its sweep index and record pointer advance in the job table, so
// replaying the same launch (a CUDA graph) continues every lattice.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "pass_bodies.cuh"

namespace cg = cooperative_groups;

namespace ising {

struct BatchJob {
    void* col0;
    void* col1;
    unsigned long long* obs;  // (E, M) slots of this launch's records; zeroed
    uint32_t thr[7];          // thresholds of the job's rule (PassArgs::thr)
    uint32_t key0, key1;
    uint32_t t0;              // index of the job's next sweep
    int32_t dims, layout, L, W;
    uint32_t rows, half;
    int32_t nsweeps, measure_every;
};

// Everything but the record slots and the sweep count, from the lattice.
static void fill_job(BatchJob& j, const ising_lattice* h, int64_t nsweeps, int every,
                     unsigned long long* obs) {
    j.col0 = h->col[0];
    j.col1 = h->col[1];
    j.obs = obs;
    rule_thresholds(h, j.thr);
    j.key0 = (uint32_t)(h->seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(h->seed >> 32);
    j.t0 = (uint32_t)h->t;
    j.dims = h->dims;
    j.layout = h->layout;
    j.L = h->L;
    j.W = h->W;
    j.rows = (uint32_t)h->rows;
    j.half = (uint32_t)h->half_sites;
    j.nsweeps = (int32_t)nsweeps;
    j.measure_every = every;
}

namespace {

constexpr int kModeCta = 0, kModeCluster = 1;

template <int MODE>
__device__ __forceinline__ void group_sync() {
    if (MODE == kModeCluster)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

// Word w of the int8 colour array when a half row holds whole words
// (W % 4 == 0): every word lies in one row, so its neighbour words are aligned
// words of the other colour -- the same word of the rows (and planes) above
// and below, and for the x-neighbours the word itself plus the previous or next
// word of its own row taken cyclically (funnel-shifted by one byte).  Every
// word, row ends and wrap rows included, takes this one path, with the rule
// and draws of int8_word (word w's draw is Philox group w).
template <int DIMS, bool MEASURE, int NC, int RULE>
__device__ __forceinline__ void int8_word_rows(const PassArgs& a, const WordGeom& g, uint32_t w,
                                               int& e_acc, int& m_neg, int& n_sites) {
    uint32_t* own = static_cast<uint32_t*>(a.own);
    const uint32_t* other = static_cast<const uint32_t*>(a.other);
    const uint32_t nq = g.W >> 2;  // words per half row
    const uint32_t r = w / nq, q = w - r * nq;
    uint32_t y = r, z = 0u;
    if (DIMS == 3) {
        z = r / g.L;
        y = r - z * g.L;
    }
    const int p = (a.c + (int)y + (int)z) & 1;
    const uint32_t row0 = r * nq;
    const uint32_t s = own[w];
    const uint32_t nx = load_other<NC>(other + w);
    uint32_t nxs;
    if (p == 0) {  // byte j <- byte j - 1 of the row, cyclically
        const uint32_t prev = load_other<NC>(other + row0 + (q == 0u ? nq - 1u : q - 1u));
        nxs = __funnelshift_l(prev, nx, 8);
    } else {       // byte j <- byte j + 1 of the row, cyclically
        const uint32_t next = load_other<NC>(other + row0 + (q + 1u == nq ? 0u : q + 1u));
        nxs = __funnelshift_r(nx, next, 8);
    }
    const uint32_t plane = z * g.L;
    const uint32_t nym = load_other<NC>(other + (plane + (y == 0u ? g.L - 1u : y - 1u)) * nq + q);
    const uint32_t nyp = load_other<NC>(other + (plane + (y + 1u == g.L ? 0u : y + 1u)) * nq + q);
    uint32_t nzm = 0u, nzp = 0u;
    if (DIMS == 3) {
        nzm = load_other<NC>(other + ((z == 0u ? g.L - 1u : z - 1u) * g.L + y) * nq + q);
        nzp = load_other<NC>(other + ((z + 1u == g.L ? 0u : z + 1u) * g.L + y) * nq + q);
    }
    const uint32_t D = disagreements<DIMS>(s, nx, nxs, nym, nyp, nzm, nzp);
    uint32_t X;
    if (RULE == kRuleHeatBath) {
        const Philox4 u = philox4x32_10(w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
        X = heatbath_count<DIMS>(D, u, a);
    } else {
        X = downhill_mask<DIMS>(D);
        if (X != 0xFEFEFEFEu) {
            const Philox4 u = philox4x32_10(w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
            X |= uphill_count<DIMS>(D, u, a);
        }
    }
    const uint32_t snew = s ^ X;
    own[w] = snew;
    if (MEASURE) {
        m_neg += __popc(snew & kByteBit7);
        n_sites += 4;
        if (a.c == 1) {
            constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
            const uint32_t Dn = (D & ~X) | ((q2 - D) & X);
            e_acc += __dp4a((int)Dn, (int)kByteOnes, 0) - 4 * 2 * DIMS;
        }
    }
}

template <int DIMS, int LAYOUT, bool MEASURE, int NC, int RULE>
__device__ __forceinline__ void job_pass(const BatchJob& j, int c, uint32_t t, uint32_t rank,
                                         uint32_t nthr, int& e_acc, int& m_acc) {
    PassArgs a;
    a.own = c == 0 ? j.col0 : j.col1;
    a.other = c == 0 ? j.col1 : j.col0;
    a.obs = nullptr;
    a.rows = j.rows;
    a.L = j.L;
    a.W = j.W;
#pragma unroll
    for (int i = 0; i < 7; ++i) a.thr[i] = j.thr[i];
    a.key0 = j.key0;
    a.key1 = j.key1;
    a.t = t;
    a.c = c;
    if (LAYOUT == ISING_INT8) {
        WordGeom g;
        g.W = (uint32_t)j.W;
        g.L = (uint32_t)j.L;
        g.rows = j.rows;
        g.half = j.half;
        const uint32_t vecs = (j.half + 15u) >> 4;
        int m_neg = 0, n_sites = 0;
        if (j.W >= 64 && vecs >= nthr) {
            for (uint32_t v = rank; v < vecs; v += nthr)
                int8_vec<DIMS, MEASURE, NC, RULE>(a, g, v, e_acc, m_neg, n_sites);
        } else if (j.W % 4 == 0 && RULE != kRuleMultiHit) {
            // short rows of whole words: one uniform path for every word
            const uint32_t words = j.half >> 2;
            for (uint32_t w = rank; w < words; w += nthr)
                int8_word_rows<DIMS, MEASURE, NC, RULE>(a, g, w, e_acc, m_neg, n_sites);
        } else {  // short rows or few vectors: four sites per item spread further
            const uint32_t words = (j.half + 3u) >> 2;
            for (uint32_t w = rank; w < words; w += nthr)
                int8_word<DIMS, MEASURE, NC, RULE>(a, g, w, e_acc, m_neg, n_sites);
        }
        if (MEASURE) m_acc += n_sites - 2 * m_neg;
    } else {
        // rows grouped by their offset in a Philox group, so that a warp's
        // words share it and take the five-call draws together
        const uint32_t items = j.rows * (((uint32_t)j.W + 31u) >> 5);
        const uint32_t rgroups = packed_row_groups((uint32_t)j.W);
        for (uint32_t it = rank; it < items; it += nthr)
            packed_word<DIMS, MEASURE, NC, RULE, RULE != kRuleMultiHit>(a, it, e_acc, m_acc,
                                                                        rgroups);
    }
}

template <int DIMS, int LAYOUT, int MODE, int RULE>
__device__ void run_job(BatchJob* jp, uint32_t rank, uint32_t nthr, bool leader) {
    // plain loads in both modes: the passes of a cluster job are separated by
    // the cluster barrier, whose release/acquire (cluster scope) makes the
    // other CTAs' writes of the previous pass visible to them (3 % faster on
    // the 2048-lattice mix than reading through L2 only)
    constexpr int NC = 0;
    const BatchJob j = *jp;
    int rec = 0;
    for (int s = 0; s < j.nsweeps; ++s) {
        const uint32_t t = j.t0 + (uint32_t)s;
        const bool measure = ((uint64_t)t + 1u) % (uint64_t)j.measure_every == 0u;
        int e = 0, m = 0;
        for (int c = 0; c < 2; ++c) {
            if (measure)
                job_pass<DIMS, LAYOUT, true, NC, RULE>(j, c, t, rank, nthr, e, m);
            else
                job_pass<DIMS, LAYOUT, false, NC, RULE>(j, c, t, rank, nthr, e, m);
            group_sync<MODE>();  // this pass's writes before the next pass reads them
        }
        if (measure) {
            block_reduce_add(e, m, j.obs + 2 * rec, true);
            ++rec;
        }
    }
    group_sync<MODE>();
    if (leader) {  // continue from here at the next launch
        jp->t0 = j.t0 + (uint32_t)j.nsweeps;
        jp->obs = j.obs + 2 * rec;
    }
}

template <int MODE, int RULE>
__device__ void dispatch_job(BatchJob* jp, uint32_t rank, uint32_t nthr, bool leader) {
    const int dims = jp->dims, layout = jp->layout;
    if (dims == 2) {
        if (layout == ISING_BITPACK)
            run_job<2, ISING_BITPACK, MODE, RULE>(jp, rank, nthr, leader);
        else
            run_job<2, ISING_INT8, MODE, RULE>(jp, rank, nthr, leader);
    } else {
        if (layout == ISING_BITPACK)
            run_job<3, ISING_BITPACK, MODE, RULE>(jp, rank, nthr, leader);
        else
            run_job<3, ISING_INT8, MODE, RULE>(jp, rank, nthr, leader);
    }
}

// counters[0] / counters[1]: next index into the large / small queue.  Every
// job of the queues uses the update rule RULE: a batch with both rules runs
// one launch per rule, so that each instance keeps its own register budget.
// 256 threads and at most 80 registers (three CTAs per SM) measured 5 % faster
// on the 2048-lattice workload than 126 registers at two per SM.  The
// heat-bath instance (every site draws, seven thresholds live) would spill at
// 80 registers, so it keeps two CTAs per SM.
template <int RULE>
__global__ void __launch_bounds__(256, RULE == kRuleHeatBath ? 2 : 3) batch_kernel(BatchJob* jobs, const int* order_big,
                                                    int n_big, const int* order_small,
                                                    int n_small, int* counters) {
    __shared__ int s_job;
    cg::cluster_group cl = cg::this_cluster();
    // phase 1: large jobs, one cluster per job
    const uint32_t crank = cl.block_rank() * blockDim.x + threadIdx.x;
    const uint32_t cthreads = cl.num_blocks() * blockDim.x;
    while (true) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) s_job = atomicAdd(&counters[0], 1);
        cl.sync();
        const int j = *cl.map_shared_rank(&s_job, 0);
        cl.sync();
        if (j >= n_big) break;
        dispatch_job<kModeCluster, RULE>(&jobs[order_big[j]], crank, cthreads, crank == 0);
    }
    // phase 2: small jobs, one CTA per job
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_job = atomicAdd(&counters[1], 1);
        __syncthreads();
        const int j = s_job;
        if (j >= n_small) break;
        dispatch_job<kModeCta, RULE>(&jobs[order_small[j]], threadIdx.x, blockDim.x,
                                     threadIdx.x == 0);
    }
}

using BatchKernel = void (*)(BatchJob*, const int*, int, const int*, int, int*);

BatchKernel batch_kernel_for(int rule) {
    return rule == kRuleHeatBath ? batch_kernel<kRuleHeatBath> : batch_kernel<kRuleMetropolis>;
}

// Resident clusters of the persistent kernel of `rule` for a launch shape.
cudaError_t resident_clusters(int rule, int threads, int cluster, int* out) {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)threads);
    cfg.gridDim = dim3((unsigned)(cluster * 1024));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(out, batch_kernel_for(rule), &cfg);
    if (e == cudaSuccess && *out < 1) return cudaErrorInvalidConfiguration;
    return e;
}

// One persistent launch over the queues of one rule.
cudaError_t launch_rule(int rule, int grid, int threads, int cluster, BatchJob* jobs,
                        const int* order, int n_big, int n_small, int* counters,
                        cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel_for(rule), jobs, order, n_big, order + n_big,
                              n_small, counters);
}

}  // namespace

}  // namespace ising

using namespace ising;

// The queues of one update rule: order[offset, offset + n_big) are the
// cluster jobs, the next n_small the per-CTA jobs.
struct RuleQueues {
    int offset = 0, n_big = 0, n_small = 0;
    int grid = 0;  // resident CTAs of that rule's kernel
};

#define ISING_BCHECK(call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ising::cuda_fail(e_); \
    } while (0)

struct ising_batch {
    std::vector<ising_lattice*> lats;
    std::vector<int64_t> sweeps;
    std::vector<int> every;
    std::vector<int> huge;  // lattices advanced by the per-lattice kernels
    std::vector<char> in_table;
    std::vector<int> order;  // per rule: [big..., small...] (host copy)
    ising_batch_opts opts{};
    cudaStream_t stream = nullptr;
    const DeviceProps* dp = nullptr;
    int cap = 0;                 // lattices the tables below can hold
    BatchJob* d_jobs = nullptr;
    BatchJob* h_jobs = nullptr;  // pinned mirror
    int* d_order = nullptr;
    int* h_order = nullptr;      // pinned mirror
    int* d_counters = nullptr;   // two per rule
    RuleQueues q[2];             // [ISING_RULE_METROPOLIS], [ISING_RULE_HEATBATH]
    int grid[2] = {0, 0};        // resident CTAs of each rule's kernel (0: not yet known)
    std::vector<int> rule;       // each lattice's rule when the batch was made
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t uploaded = nullptr;
    bool table_valid = false;  // device table equals the host mirror's continuation
    bool order_dirty = true;   // the device order array must be uploaded
    int64_t launches = 0;
};

namespace {

int records_in(uint64_t t, int64_t n, int every) {
    return (int)((t + (uint64_t)n) / (uint64_t)every - t / (uint64_t)every);
}

cudaError_t launch_batch_kernel(ising_batch* b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, 4 * sizeof(int), st);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        const RuleQueues& q = b->q[r];
        if (q.n_big + q.n_small == 0) continue;
        e = launch_rule(r, q.grid, b->opts.block_threads, b->opts.cluster_size, b->d_jobs,
                        b->d_order + q.offset, q.n_big, q.n_small, b->d_counters + 2 * r, st);
    }
    return e;
}

int queued_jobs(const ising_batch* b) {
    return b->q[0].n_big + b->q[0].n_small + b->q[1].n_big + b->q[1].n_small;
}

void free_batch(ising_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->uploaded) cudaEventDestroy(b->uploaded);
    if (b->d_jobs) cudaFreeAsync(b->d_jobs, b->stream);
    if (b->d_order) cudaFreeAsync(b->d_order, b->stream);
    if (b->d_counters) cudaFreeAsync(b->d_counters, b->stream);
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->h_order) cudaFreeHost(b->h_order);
    delete b;
}

// Arguments of a batch's lattice list: valid handles, each at most once.
int check_members(ising_lattice* const* lats, int n, const int64_t* sweeps,
                  const int* measure_every) {
    if (!lats || n < 1 || !sweeps) return ISING_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!lats[i] || sweeps[i] < 0 || sweeps[i] > 0x7FFFFFFF) return ISING_EINVAL;
        if (measure_every && measure_every[i] < 1) return ISING_EINVAL;
    }
    std::vector<ising_lattice*> sorted(lats, lats + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return ISING_EINVAL;  // a lattice may appear once
    return ISING_OK;
}

// Take a new lattice list: move the lattices to the batch stream, build the
// per-rule queues (largest work first, split at the size thresholds) and make
// room in the tables.  Growing the tables frees the old ones in stream order,
// after any launch already queued.
int assign_members(ising_batch* b, ising_lattice* const* lats, int n, const int64_t* sweeps,
                   const int* measure_every) {
    const ising_batch_opts& o = b->opts;
    for (int i = 0; i < n; ++i) {
        const int rc = ising_set_stream(lats[i], b->stream);
        if (rc != ISING_OK) return rc;
    }
    b->lats.assign(lats, lats + n);
    b->sweeps.assign(sweeps, sweeps + n);
    b->every.resize(n);
    for (int i = 0; i < n; ++i) b->every[i] = measure_every ? measure_every[i] : 1;
    std::vector<int> big[2], small[2];
    b->huge.clear();
    b->in_table.assign(n, 1);
    b->rule.resize(n);
    for (int i = 0; i < n; ++i) {
        const int r = b->lats[i]->rule == ISING_RULE_HEATBATH ? 1 : 0;
        b->rule[i] = b->lats[i]->rule;
        // the largest lattices, and the rules without a persistent-kernel form
        // (demon dynamics, multi-hit), go through the per-lattice kernels
        if ((o.huge_sites > 0 && b->lats[i]->sites >= o.huge_sites) ||
            b->lats[i]->rule == ISING_RULE_DEMON || b->lats[i]->rule == ISING_RULE_MULTIHIT) {
            b->huge.push_back(i);
            b->in_table[i] = 0;
        } else {
            (o.cluster_size > 1 && b->lats[i]->sites >= o.big_sites ? big[r] : small[r])
                .push_back(i);
        }
    }
    auto by_work = [&](int x, int y) {
        return b->lats[x]->sites * b->sweeps[x] > b->lats[y]->sites * b->sweeps[y];
    };
    b->order.clear();
    for (int r = 0; r < 2; ++r) {
        std::stable_sort(big[r].begin(), big[r].end(), by_work);
        std::stable_sort(small[r].begin(), small[r].end(), by_work);
        b->q[r].offset = (int)b->order.size();
        b->q[r].n_big = (int)big[r].size();
        b->q[r].n_small = (int)small[r].size();
        b->order.insert(b->order.end(), big[r].begin(), big[r].end());
        b->order.insert(b->order.end(), small[r].begin(), small[r].end());
    }
    if (n > b->cap) {
        // the pinned mirrors may still be the source of a queued upload
        if (b->uploaded) ISING_BCHECK(cudaEventSynchronize(b->uploaded));
        if (b->d_jobs) ISING_BCHECK(cudaFreeAsync(b->d_jobs, b->stream));
        if (b->d_order) ISING_BCHECK(cudaFreeAsync(b->d_order, b->stream));
        if (b->h_jobs) ISING_BCHECK(cudaFreeHost(b->h_jobs));
        if (b->h_order) ISING_BCHECK(cudaFreeHost(b->h_order));
        b->d_jobs = nullptr;
        b->d_order = nullptr;
        b->h_jobs = nullptr;
        b->h_order = nullptr;
        b->cap = 0;
        const int cap = n;
        ISING_BCHECK(pool_alloc(reinterpret_cast<void**>(&b->d_jobs), sizeof(BatchJob) * cap,
                                *b->dp, b->stream));
        ISING_BCHECK(pool_alloc(reinterpret_cast<void**>(&b->d_order), sizeof(int) * cap,
                                *b->dp, b->stream));
        ISING_BCHECK(cudaMallocHost(reinterpret_cast<void**>(&b->h_jobs), sizeof(BatchJob) * cap));
        ISING_BCHECK(cudaMallocHost(reinterpret_cast<void**>(&b->h_order), sizeof(int) * cap));
        b->cap = cap;
    }
    // persistent grids: as many clusters as can be resident (once per rule)
    for (int r = 0; r < 2; ++r) {
        if (b->q[r].n_big + b->q[r].n_small == 0 || b->grid[r] > 0) {
            b->q[r].grid = b->grid[r];
            continue;
        }
        int clusters = 0;
        ISING_BCHECK(resident_clusters(r, o.block_threads, o.cluster_size, &clusters));
        b->grid[r] = clusters * o.cluster_size;
        b->q[r].grid = b->grid[r];
    }
    if (b->exec) {  // the captured launch holds the old queue sizes
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->table_valid = false;
    b->order_dirty = true;
    return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_create(ising_batch** out, ising_lattice* const* lats, int n,
                       const int64_t* sweeps, const int* measure_every,
                       const ising_batch_opts* opts, void* stream) {
    if (!out) return ISING_EINVAL;
    *out = nullptr;
    ising_batch_opts o = {};
    if (opts) o = *opts;
    if (o.block_threads == 0) o.block_threads = 256;
    if (o.cluster_size == 0) o.cluster_size = 4;
    if (o.big_sites == 0) o.big_sites = 1 << 18;
    if (o.huge_sites == 0) o.huge_sites = (int64_t)1 << 22;
    if (o.block_threads != 128 && o.block_threads != 256) return ISING_EINVAL;
    if (o.cluster_size < 1 || o.cluster_size > 8) return ISING_EINVAL;
    int rc = check_members(lats, n, sweeps, measure_every);
    if (rc != ISING_OK) return rc;
    const DeviceProps* dp = nullptr;
    rc = device_props(&dp);
    if (rc != ISING_OK) return rc;
    ising_batch* b = new (std::nothrow) ising_batch();
    if (!b) return ISING_ENOMEM;
    b->opts = o;
    b->dp = dp;
    b->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = pool_alloc(reinterpret_cast<void**>(&b->d_counters), 4 * sizeof(int), *dp,
                               b->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e);
    }
    rc = assign_members(b, lats, n, sweeps, measure_every);
    if (rc != ISING_OK) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return ISING_OK;
}

int ising_batch_update(ising_batch* b, ising_lattice* const* lats, int n, const int64_t* sweeps,
                       const int* measure_every) {
    if (!b) return ISING_EINVAL;
    const int rc = check_members(lats, n, sweeps, measure_every);
    if (rc != ISING_OK) return rc;
    return assign_members(b, lats, n, sweeps, measure_every);
}

int ising_batch_launch(ising_batch* b) {
    if (!b) return ISING_EINVAL;
    const int n = (int)b->lats.size();
    // host-side checks and record space, then the job table if it changed
    bool moved = !b->table_valid;
    for (int i = 0; i < n; ++i) {
        ising_lattice* h = b->lats[i];
        if (b->sweeps[i] > 0 && h->t + (uint64_t)b->sweeps[i] - 1 > kMaxSweep) return ISING_ERANGE;
        if (h->rule != b->rule[i]) return ISING_EINVAL;  // queues are per rule, fixed at create
    }
    // the largest lattices first, each pass over the whole GPU
    for (int i : b->huge) {
        const int rc = ising_sweep(b->lats[i], b->sweeps[i], b->every[i]);
        if (rc != ISING_OK) return rc;
    }
    ISING_BCHECK(cudaEventSynchronize(b->uploaded));  // the mirrors are free to change
    for (int i = 0; i < n; ++i) {
        if (!b->in_table[i]) continue;
        ising_lattice* h = b->lats[i];
        const int r = records_in(h->t, b->sweeps[i], b->every[i]);
        unsigned long long* before = h->obs;
        // keep room for several launches so that replays need no new table
        int rc = ensure_records(h, h->n_rec + 8 * (int64_t)(r > 0 ? r : 0));
        if (rc != ISING_OK) return rc;
        if (h->obs != before) moved = true;
        fill_job(b->h_jobs[i], h, b->sweeps[i], b->every[i], h->obs + 2 * h->n_rec);
    }
    // records reserved for later launches must stay inside the capacity: if the
    // last reserve is about to run out, the table is rebuilt (moved == true)
    if (moved || b->order_dirty) {
        ISING_BCHECK(cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(BatchJob) * (size_t)n,
                                     cudaMemcpyHostToDevice, b->stream));
        if (b->order_dirty && !b->order.empty()) {  // empty when every lattice is huge
            std::memcpy(b->h_order, b->order.data(), sizeof(int) * b->order.size());
            ISING_BCHECK(cudaMemcpyAsync(b->d_order, b->h_order, sizeof(int) * b->order.size(),
                                         cudaMemcpyHostToDevice, b->stream));
        }
        ISING_BCHECK(cudaEventRecord(b->uploaded, b->stream));
        b->table_valid = true;
        b->order_dirty = false;
    }
    if (b->opts.use_graph >= 0 && !b->exec && queued_jobs(b) > 0) {
        // capture [reset queue counters, persistent kernel] once; replay it
        cudaStream_t cap = nullptr;
        ISING_BCHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = launch_batch_kernel(b, cap);
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (queued_jobs(b) > 0) {
        if (b->exec)
            ISING_BCHECK(cudaGraphLaunch(b->exec, b->stream));
        else
            ISING_BCHECK(launch_batch_kernel(b, b->stream));
    }
    for (int i = 0; i < n; ++i) {
        if (!b->in_table[i]) continue;
        ising_lattice* h = b->lats[i];
        h->n_rec += records_in(h->t, b->sweeps[i], b->every[i]);
        h->t += (uint64_t)b->sweeps[i];
    }
    // the device table now holds the continuation; it stays valid while no
    // lattice's record buffer moves and nothing else touches the lattices
    ++b->launches;
    return ISING_OK;
}

int ising_batch_sync(ising_batch* b) {
    if (!b) return ISING_EINVAL;
    ISING_BCHECK(cudaStreamSynchronize(b->stream));
    b->table_valid = false;  // lattices may now be used directly; rebuild next time
    return ISING_OK;
}

void ising_batch_destroy(ising_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
}

int ising_batch_run(ising_lattice* const* lats, int n, const int64_t* sweeps, int measure_every,
                    void* stream) {
    if (measure_every < 1 || n < 1) return ISING_EINVAL;
    std::vector<int> every;
    try {
        every.assign((size_t)n, measure_every);
    } catch (const std::bad_alloc&) {
        return ISING_ENOMEM;
    }
    // one launch: a plain launch rather than a graph captured for one replay
    ising_batch_opts o = {};
    o.use_graph = -1;
    ising_batch* b = nullptr;
    int rc = ising_batch_create(&b, lats, n, sweeps, every.data(), &o, stream);
    if (rc != ISING_OK) return rc;
    rc = ising_batch_launch(b);
    const int rs = ising_batch_sync(b);
    ising_batch_destroy(b);
    return rc != ISING_OK ? rc : rs;
}

int ising_batch_info(const ising_batch* b, int* grid, int* n_big, int* n_small, int* n_huge) {
    if (!b) return ISING_EINVAL;
    if (grid) *grid = b->q[0].grid > b->q[1].grid ? b->q[0].grid : b->q[1].grid;
    if (n_big) *n_big = b->q[0].n_big + b->q[1].n_big;
    if (n_small) *n_small = b->q[0].n_small + b->q[1].n_small;
    if (n_huge) *n_huge = (int)b->huge.size();
    return ISING_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// The batched launch without allocation.  For callers that must not allocate
// device memory once they are running (a real-time loop, a process that owns
// a fixed memory pool, code that runs where cudaMalloc would synchronise or
// fail), the job table, the queue order and the queue counters live in one
// file-scope device array of fixed size instead of in memory the library
// allocates; the caller's lattices and record buffer are the only other
// memory touched.
// ----------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxJobs = 2048;
constexpr size_t kStaticTableBytes = sizeof(BatchJob) * kStaticMaxJobs;
constexpr size_t kStaticOrderBytes = sizeof(int) * kStaticMaxJobs;
static_assert(sizeof(BatchJob) == 96, "the scratch size quoted in ising.h assumes 96-byte jobs");

// job table | order | queue counters; every GPU that loads the library holds
// it (about 200 KiB) until the process exits
static __device__ __align__(256) unsigned char g_static_scratch[kStaticTableBytes +
                                                                  kStaticOrderBytes + 256];

struct StaticSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    int clusters[2][2][9] = {};        // resident clusters per [rule][block size][cluster size]
};
std::mutex g_static_mu;
StaticSetup g_static[64];

int block_index(int threads) { return threads == 128 ? 0 : 1; }

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in for it) and, once per
// rule and launch shape, the resident grid size.  Neither call allocates.
int static_setup(int threads, int cluster, unsigned char** scratch, int grid[2]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return ISING_ECUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticSetup& st = g_static[dev];
    if (!st.ready) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        st.scratch = static_cast<unsigned char*>(ptr);
        st.ready = true;
    }
    for (int r = 0; r < 2; ++r) {
        int& c = st.clusters[r][block_index(threads)][cluster];
        if (c < 1) {
            int nc = 0;
            e = resident_clusters(r, threads, cluster, &nc);
            if (e != cudaSuccess) return cuda_fail(e);
            c = nc;
        }
        grid[r] = c * cluster;
    }
    *scratch = st.scratch;
    return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_run_static(ising_lattice* const* lats, int n, const int64_t* sweeps,
                           const int* measure_every, int64_t* records, int64_t records_cap,
                           const ising_batch_opts* opts, void* stream) {
    if (!lats || !sweeps || n < 1) return ISING_EINVAL;
    if (n > kStaticMaxJobs) return ISING_ERANGE;  // more lattices than the fixed job table holds
    ising_batch_opts o = {};
    if (opts) o = *opts;
    if (o.block_threads == 0) o.block_threads = 256;
    if (o.cluster_size == 0) o.cluster_size = 4;
    if (o.big_sites == 0) o.big_sites = 1 << 18;
    if (o.block_threads != 128 && o.block_threads != 256) return ISING_EINVAL;
    if (o.cluster_size < 1 || o.cluster_size > 8) return ISING_EINVAL;
    // validate everything and count the records before touching the GPU
    int64_t total_rec = 0;
    for (int i = 0; i < n; ++i) {
        const ising_lattice* h = lats[i];
        if (!h || sweeps[i] < 0 || sweeps[i] > 0x7FFFFFFF) return ISING_EINVAL;
        if (h->rule == ISING_RULE_DEMON || h->rule == ISING_RULE_MULTIHIT)
            return ISING_EINVAL;  // not in the persistent kernel
        // stream order is the only ordering against the handle's own work
        // (earlier sweeps, later reads): the lattice must already be on `stream`
        if (h->stream != static_cast<cudaStream_t>(stream)) return ISING_EINVAL;
        const int every = measure_every ? measure_every[i] : 1;
        if (every < 1) return ISING_EINVAL;
        if (sweeps[i] > 0 && h->t + (uint64_t)sweeps[i] - 1 > kMaxSweep) return ISING_ERANGE;
        for (int k = 0; k < i; ++k)
            if (lats[k] == h) return ISING_EINVAL;
        total_rec += records_in(h->t, sweeps[i], every);
    }
    if (total_rec > 0 && (!records || records_cap < total_rec)) return ISING_ERANGE;
    unsigned char* scratch = nullptr;
    int grid[2] = {0, 0};
    int rc = static_setup(o.block_threads, o.cluster_size, &scratch, grid);
    if (rc != ISING_OK) return rc;
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    BatchJob* d_jobs = reinterpret_cast<BatchJob*>(scratch);
    int* d_order = reinterpret_cast<int*>(scratch + kStaticTableBytes);
    int* d_counters = reinterpret_cast<int*>(scratch + kStaticTableBytes + kStaticOrderBytes);

    // queues per rule, largest work first: cluster-cooperative jobs, then
    // per-CTA jobs (the same order as ising_batch_create)
    int order[kStaticMaxJobs];
    int off[3] = {0, 0, 0}, n_big[2] = {0, 0};
    auto work = [&](int i) { return lats[i]->sites * sweeps[i]; };
    auto by_work = [&](int x, int y) { return work(x) > work(y); };
    int n_all = 0;
    for (int r = 0; r < 2; ++r) {
        off[r] = n_all;
        for (int pass = 0; pass < 2; ++pass) {
            const int begin = n_all;
            for (int i = 0; i < n; ++i) {
                const bool big = o.cluster_size > 1 && lats[i]->sites >= o.big_sites;
                if ((lats[i]->rule == ISING_RULE_HEATBATH ? 1 : 0) == r && big == (pass == 0))
                    order[n_all++] = i;
            }
            std::stable_sort(order + begin, order + n_all, by_work);
            if (pass == 0) n_big[r] = n_all - begin;
        }
    }
    off[2] = n_all;

    cudaError_t e = cudaSuccess;
    if (total_rec > 0)  // the fused reductions add into zeroed record slots
        e = cudaMemsetAsync(records, 0, (size_t)total_rec * 16, sm);
    // job table, staged through a small host buffer (copies from pageable
    // memory are complete as far as the source is concerned on return)
    constexpr int kChunk = 32;
    BatchJob chunk[kChunk];
    int64_t rec_off = 0;
    for (int base = 0; base < n && e == cudaSuccess; base += kChunk) {
        const int m = n - base < kChunk ? n - base : kChunk;
        for (int q = 0; q < m; ++q) {
            const int i = base + q;
            const ising_lattice* h = lats[i];
            const int every = measure_every ? measure_every[i] : 1;
            fill_job(chunk[q], h, sweeps[i], every,
                     reinterpret_cast<unsigned long long*>(records) + 2 * rec_off);
            rec_off += records_in(h->t, sweeps[i], every);
        }
        e = cudaMemcpyAsync(d_jobs + base, chunk, sizeof(BatchJob) * (size_t)m,
                            cudaMemcpyHostToDevice, sm);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_order, order, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counters, 0, 4 * sizeof(int), sm);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        const int jobs = off[r + 1] - off[r];
        if (jobs == 0) continue;
        e = launch_rule(r, grid[r], o.block_threads, o.cluster_size, d_jobs, d_order + off[r],
                        n_big[r], jobs - n_big[r], d_counters + 2 * r, sm);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < n; ++i) lats[i]->t += (uint64_t)sweeps[i];
    return ISING_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Small lattices through ising_sweep: with a few thousand sites a colour pass
// lasts less than its launch, so n sweeps run as one job on a single CTA (the
// same arithmetic and draws; passes separated by __syncthreads) instead of 2n
// launches.  The job travels by value and lives in shared memory.
// ----------------------------------------------------------------------------
namespace ising {

namespace {

template <int RULE>
__global__ void __launch_bounds__(256, 1) small_job_kernel(BatchJob job) {
    __shared__ BatchJob sj;
    if (threadIdx.x == 0) sj = job;
    __syncthreads();
    dispatch_job<kModeCta, RULE>(&sj, threadIdx.x, blockDim.x, threadIdx.x == 0);
}

}  // namespace

int small_sweep(ising_lattice* h, int64_t n, int every, unsigned long long* slots) {
    BatchJob j;
    fill_job(j, h, n, every, slots);
    if (h->rule == ISING_RULE_HEATBATH)
        small_job_kernel<kRuleHeatBath><<<1, 256, 0, h->stream>>>(j);
    else
        small_job_kernel<kRuleMetropolis><<<1, 256, 0, h->stream>>>(j);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : cuda_fail(e);
}

}  // namespace ising
