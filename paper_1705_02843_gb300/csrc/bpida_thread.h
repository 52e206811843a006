// Internal interface of the thread-parallel IDA* ablations and of the paper's
// BPIDA* with its static load balancing (bpida_thread.cu), reached through
// bpida_solve_ex with variant = 2, 3, 4 or 5.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpida.h"

namespace bp {
namespace tp {

enum { PSIMPLE = 2, PSTATICLB = 3, PFULLLB = 4, BPSTATIC = 5 };

struct Settings {
    int width;    // 3 or 4
    int variant;  // PSIMPLE, PSTATICLB, PFULLLB or BPSTATIC
    int threads;  // search threads (BPSTATIC: warps); 0 = all resident ones of the search kernel
};

// Solves the n boards one after another (one instance per run, as in the
// paper's experiments); outputs as bpida_solve_ex. Fills the thread-parallel
// fields of *stats (and the common ones it can).
bpida_status solve(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                   uint64_t *out_nodes, int *out_iters, int *out_status, uint64_t *out_solutions, cudaStream_t st,
                   bpida_stats *stats);

// Frees the calling device's thread-parallel workspace.
void release(int dev);

}  // namespace tp
}  // namespace bp
