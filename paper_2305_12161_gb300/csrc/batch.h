// Work list of the batched persistent kernel (k_batch.cu) and its host launcher.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

constexpr int BATCH_THREADS = 256;
constexpr int BATCH_LOCAL = 0;   // CTA owns whole lattices, kept in shared memory
constexpr int BATCH_GROUP = 1;   // CTA is one rank of a group sharing a lattice
constexpr int BATCH_STATUS_TIMEOUT = 1;

struct BatchLattice {
    uint32_t *lat;  // 2 * nw words: sublattice 0 then 1
    uint64_t S;     // Philox key: seed + replica
    int L;
    int pad;
};

struct BatchTask {
    int mode;   // BATCH_LOCAL or BATCH_GROUP
    int first;  // LOCAL: first lattice index; GROUP: the lattice index
    int count;  // LOCAL: number of lattices (consecutive)
    int group;  // GROUP: barrier counter index
    int rank;   // GROUP: rank in group
    int size;   // GROUP: CTAs in group
};

cudaError_t batch_occupancy(int smem_bytes, int *blocks_per_sm);

cudaError_t launch_batch(const BatchTask *tasks, int ntasks, const BatchLattice *lats, int rule, uint32_t t0,
                         int n_mcs, unsigned *barriers, int *status, uint64_t timeout_ns, int missing_cta,
                         unsigned long long *cta_ns, int smem_bytes, cudaStream_t s);

}  // namespace ising
