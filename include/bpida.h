/*
 * bpida.h — C ABI of the GB300 (sm_103a) Block-Parallel IDA* solver.
 *
 * The solver finds optimal solutions of sliding-tile puzzles (8-, 15- and
 * 24-puzzle) with IDA* under the Manhattan distance heuristic, running the
 * f-limited depth-first search of every iteration on the GPU with a warp
 * per subtree (Horie & Fukunaga, "Block-Parallel IDA* for GPUs",
 * Section 5, Algorithm 1). All integer results are exact.
 *
 * Conventions (every buffer and result uses them):
 *   - positions are row-major 0 .. W*W-1; the goal has tile t at position t
 *     and the blank (tile 0) at position 0;
 *   - a move is the direction the blank travels: 0 = up, 1 = left,
 *     2 = right, 3 = down; the inverse of the previous move is never
 *     applied;
 *   - a node is counted ("expanded") when it is taken off the search stack
 *     with f <= limit; the root and goal nodes count; a goal is not
 *     expanded further;
 *   - the first f-limit is h(start); each later limit is the smallest f of
 *     the children pruned in the previous iteration (Algorithm 1);
 *   - with count_all = 1 the final iteration is searched to completion, as
 *     in the all-optimal-solutions experiment of Section 6, so its node
 *     count does not depend on the order in which nodes are expanded, and
 *     the solution returned is the lexicographically first optimal one;
 *   - with count_all = 0 (first-solution mode, Section 6's main timing
 *     experiment) an instance stops as soon as one of its warps pops a goal:
 *     the non-final iterations' counts are unchanged, the final iteration's
 *     count is what was expanded before the stop (it depends on timing; at
 *     most the count_all = 1 count, which it equals when a call of at most 8
 *     boards searched that iteration in one step with the ones before it),
 *     and the solution returned is an optimal one, not necessarily the
 *     first.
 *
 * Board packing (device memory, read-only to the library):
 *   W = 3 or 4: one uint64_t per board, tile at position p in bits [4p, 4p+4).
 *   W = 5:      two uint64_t per board (low word first) forming a 128-bit
 *               integer with the tile at position p in bits [5p, 5p+5).
 *
 * Streams and ownership: every pointer argument of the solve calls is
 * DEVICE memory owned by the caller; the library keeps no reference after
 * the call's work has finished. The solve calls are stream-ordered and
 * asynchronous: with the default driver (driver = 0) a call enqueues its
 * work on `stream` and returns without waiting for it; the inputs must stay
 * valid and the outputs untouched until the stream has reached the end of
 * the call's work (synchronise the stream, or order later work after it).
 * Calls on the same stream run one after another; calls on different
 * streams may overlap on the device. Each call takes a workspace from a
 * per-device pool of at most four (grown on demand, freed by
 * bpida_release_workspace()): the one last used on the same stream, else
 * an idle one, else a new one; with four busy on other streams the call's
 * stream waits on the device for the least recently used one. The first
 * call with a new configuration or a larger batch may allocate device
 * memory and build a CUDA graph, and a call that has to grow a busy
 * workspace waits for that workspace's last call first. The host-driven
 * loop (driver = 1), the ablation variants 2-5 and
 * bpida_solve_noalloc synchronise `stream` before returning. The library
 * serialises its host-side bookkeeping with a process-wide lock, held while
 * a call is enqueued.
 *
 * Errors: arguments the host can check are rejected synchronously with
 * BPIDA_EINVAL before any work is issued, and a failed CUDA runtime call
 * returns BPIDA_ECUDA (BPIDA_ENOMEM for a failed allocation). What the
 * device finds is reported per instance once the work has finished:
 * out_status[i] (bpida_solve_ex) and out_len[i] = -1 for an unsolvable
 * board, a node budget or length cap that ran out, and, for every instance
 * not finished when a call-wide problem stopped the search (hand-back
 * queue capacity: BPIDA_ENOMEM; a failed internal check: BPIDA_EINTERNAL),
 * that problem. Per-instance problems do not stop the other instances. The
 * library never calls __trap() or a device assert.
 */
#ifndef BPIDA_H
#define BPIDA_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BPIDA_OK = 0,
    BPIDA_EINVAL = 1,   /* bad argument, or a board that is not a permutation
                           or not in the goal's parity class (unsolvable) */
    BPIDA_ENOMEM = 2,   /* device workspace or work-queue capacity exceeded */
    BPIDA_ESTACK = 3,   /* reserved: search stack bound exceeded */
    BPIDA_EBUDGET = 4,  /* node budget exhausted before a solution */
    BPIDA_ETIMEOUT = 5, /* reserved: a bounded device wait gave up */
    BPIDA_ECUDA = 6,    /* a CUDA runtime call failed */
    BPIDA_ELIMIT = 7,   /* solution longer than bpida_max_len(width) */
    BPIDA_EINTERNAL = 8 /* an internal consistency check failed */
} bpida_status;

typedef struct {
    int width;            /* 3, 4 or 5 (8-, 15-, 24-puzzle); 0 means 4 */
    int count_all;        /* 1 = final iteration searched to completion,
                             0 = stop at the first solution found */
    int split_target;     /* max frontier records per instance; 0 = auto */
    int warps_per_block;  /* search kernel block size in warps; 0 = auto */
    int stack_entries;    /* per-warp shared-memory stack, 0 = auto
                             (width 4 and 5: 384, 3: 512); one of 256,
                             384, 480, 512, 768, 1024. Smaller stacks
                             spill to the hand-back queue more often: with
                             256 a batch of hard boards can overflow it
                             (those instances end with BPIDA_ENOMEM) */
    int exit_fraction_pct;/* percentage of warps that must have run out of
                             work before busy warps hand their stacks back
                             for redistribution; 0 = auto */
    int min_rounds;       /* rounds a warp runs before it may hand back its
                             stack; 0 = auto */
    uint64_t node_budget; /* per instance, over all iterations; 0 = none */
    int driver;           /* 0 = the threshold loop runs as one CUDA graph
                             with device-set loop conditions (default);
                             1 = the host launches every kernel and reads
                             the loop state back after every search pass
                             (needed for per-launch CUDA-event timing) */
    int min_pass_us;      /* a pass hands work back only after running this
                             long (microseconds); 0 = auto, -1 = no minimum */
    int variant;          /* search kernel: 0 = warp per subtree group, one
                             node per lane, work queue and hand-back
                             (default); 1 = the paper's BPIDA* kernel
                             (Algorithm 1: block = warp, 8 nodes per pop,
                             lane i applies action i mod 4, roots assigned
                             statically, no dynamic load balancing) on this
                             design's per-iteration root sets, kept as an
                             ablation; 2, 3, 4 = the paper's thread-
                             parallel configurations PSimple, PStaticLB and
                             PFullLB (Section 4 and its appendix: one
                             sequential depth-first search per thread over
                             the roots assigned to it; no load balancing /
                             static rebalancing of a persistent root set by
                             the previous iteration's per-root loads / the
                             same plus idle threads taking untried branches
                             from busy threads of their block); 5 = the
                             paper's BPIDA* with its own static load
                             balancing (Section 5: variant 1's warp search
                             over a persistent root set that is split and
                             reassigned after every iteration by the
                             repetitions each root took, as PStaticLB does
                             with node counts), all kept as ablations.
                             Variants 2-5 take width 3 or 4, count_all = 1
                             and no node budget (else BPIDA_EINVAL), solve
                             the boards one at a time, synchronise the
                             stream, use split_target as the number of
                             search threads (variant 5: warps; 0 = every
                             resident one) and report the load balance in
                             bpida_stats; their solution is an optimal one
                             (for 2, 3 and 5 the lexicographically first),
                             and every count equals variant 0's; 6 = block
                             per subtree group: variant 0's queue and
                             hand-back, but the warps of a block share one
                             stack (warps_per_block x stack_entries
                             entries), a round pops one node per thread,
                             and children are placed by a block-wide prefix
                             (the autotuner's other mode; width 3 or 4, one
                             iteration per step) */
    int reserved;
} bpida_config;

typedef struct {
    int steps;              /* device steps issued (all instances); a call of
                               at most 8 boards without a node budget may
                               search several consecutive thresholds of an
                               instance in one step, with the same
                               per-iteration results */
    int passes;             /* search kernel launches */
    uint64_t records;       /* frontier records produced by the splitter */
    uint64_t handed_back;   /* stack entries handed back between passes */
    uint64_t search_nodes;  /* nodes expanded inside the search kernel */
    double search_ms;       /* sum of search kernel durations from CUDA
                               events on the launching stream; only with
                               bpida_set_timing(1) and driver = 1 */
    int grid_blocks;        /* search kernel grid */
    int block_threads;      /* search kernel block */
    int sm_count;
    int launches;           /* kernels launched by the call */
    uint64_t spills;        /* stack overflows handed to the next pass */
    int max_handed_back;    /* largest hand-back queue of one pass */
    double search_ms_device;/* sum of search kernel durations measured on
                               the device (first block start to last block
                               end, %globaltimer), any driver */
    /* variants 2-5 only, zero otherwise: */
    int tp_threads;         /* search threads (variant 5: search warps) */
    int tp_pad;
    double lb_ratio;        /* load balance of the last board's next-to-last
                               iteration (its only one if it had one): the
                               largest per-thread (variant 5: per-warp) node
                               count over the mean over all of them */
    double lb_ratio_last;   /* the same for its final iteration */
    uint64_t tp_roots;      /* roots in the last board's final root set */
    uint64_t tp_balances;   /* variant 4: in-block balancing operations */
    uint64_t tp_steals;     /* variant 4: branches moved to idle threads */
} bpida_stats;

/* Upper bounds used to size the per-instance output rows. */
int bpida_max_len(int width);    /* moves per solution row */
int bpida_max_iters(int width);  /* iterations per node-count row */

/*
 * Solve n boards with the default configuration (15-puzzle, count_all = 1).
 *   boards             device, n words (packing above)
 *   out_len            device, n ints: optimal length, -1 if none
 *   out_moves          device, n * bpida_max_len(4) bytes; row i holds the
 *                      lexicographically first optimal solution (moves in
 *                      the order up < left < right < down), zero-filled
 *   out_nodes_per_iter device, n * bpida_max_iters(4) uint64: nodes
 *                      expanded in each iteration, zero-filled
 * Returns BPIDA_OK once the work is enqueued on `stream` (the results are
 * written when the stream reaches the end of it), or the error of a call
 * that could not be issued (a bad argument, a CUDA error, device memory).
 * An instance with out_len -1 was not solved (its reason is its
 * bpida_solve_ex out_status entry).
 */
bpida_status bpida_solve(const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                         uint64_t *out_nodes_per_iter, void *stream);

/*
 * As bpida_solve, with a configuration and per-instance outputs:
 *   out_num_iters device, n ints: iterations run (may be NULL)
 *   out_status    device, n ints: bpida_status of each instance (may be NULL)
 *   out_solutions device, n uint64: goals popped in the final iteration, i.e.
 *                 with count_all = 1 the number of optimal solutions (move
 *                 sequences of optimal length that never undo the previous
 *                 move); with count_all = 0 at least 1 (may be NULL)
 * Row widths are bpida_max_len(cfg->width) and bpida_max_iters(cfg->width).
 */
bpida_status bpida_solve_ex(const bpida_config *cfg, const uint64_t *boards, int n, int *out_len,
                            uint8_t *out_moves, uint64_t *out_nodes_per_iter, int *out_num_iters,
                            int *out_status, uint64_t *out_solutions, void *stream);

/*
 * bpida_solve_noalloc — the 15-puzzle solve without any device allocation.
 * The paper has no counterpart: it serves callers that cannot call
 * cudaMalloc when they want a solve (a device whose memory a framework's
 * pool allocator has already reserved, loops that cannot take cudaMalloc's
 * implicit device synchronisation).
 *   Same arguments and results as bpida_solve_ex with the default
 *   configuration (width 4, count_all = 1): boards, out_len, out_moves
 *   (n * bpida_max_len(4) bytes), out_nodes_per_iter (n * bpida_max_iters(4)
 *   uint64), out_num_iters and out_status (may be NULL) are caller-owned
 *   device buffers.
 *   n may be at most BPIDA_NOALLOC_MAX_BOARDS; a larger n returns
 *   BPIDA_EINVAL before any work is issued.
 *   The workspace is one file-scope __device__ array of
 *   BPIDA_NOALLOC_SCRATCH_BYTES held by every GPU that loads the library
 *   until the process exits. The first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current;
 *   after a cudaDeviceReset, call bpida_release_workspace() (which forgets
 *   the address) before the next call. No call allocates or frees memory.
 *   Calls share the array: each call re-initialises what it reads, and calls
 *   that overlapped on the GPU would race (calls are serialised by a lock
 *   and synchronise `stream` before returning). The search runs with one
 *   two-warp block per SM, so it is slower than bpida_solve_ex; a hand-back
 *   overflow of its fixed queue (2^18 records per pass) returns
 *   BPIDA_ENOMEM.
 */
#define BPIDA_NOALLOC_MAX_BOARDS 256
#define BPIDA_NOALLOC_SCRATCH_BYTES (16u << 20)
bpida_status bpida_solve_noalloc(const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                                 uint64_t *out_nodes_per_iter, int *out_num_iters, int *out_status,
                                 void *stream);

/*
 * Serving: a continuous-batching solve service for the 15-puzzle (the
 * paper solves one instance per run; this is the batched solver kept
 * running). Requests are submitted one board at a time from host memory at
 * any moment; a background host thread admits them into free instance slots
 * between threshold steps, so newly arrived requests share every search
 * pass with those already on the GPU, each with its own f-limit. Search
 * state stays in device memory across thresholds. Results (the same as
 * bpida_solve_ex gives for that board alone: all-solutions node counts, the
 * lexicographically first optimal solution) are posted to a completion
 * queue as soon as the request finishes.
 */
typedef struct bpida_server bpida_server;

typedef struct {
    uint64_t req_id;
    int status;                 /* bpida_status of the request */
    int length;                 /* optimal length, -1 if none */
    int num_iters;              /* iterations run */
    int pad;
    double submit_time_s;       /* bpida_server_clock() at submit */
    double done_time_s;         /* bpida_server_clock() when it became pollable */
    uint8_t moves[80];          /* first optimal solution, zero-filled */
    uint64_t nodes_per_iter[41];/* nodes expanded per iteration, zero-filled */
    uint64_t solutions;         /* number of optimal solutions */
} bpida_result;

typedef struct {
    int slots;                  /* instance slots (bounded by frontier memory) */
    int max_active;             /* most instances searched in one step */
    uint64_t submitted, admitted, completed;
    uint64_t steps, passes;     /* device threshold steps and search passes */
    uint64_t sliced_steps;      /* steps cut by the time slice (open nodes
                                   carried into the next step) */
} bpida_server_stats;

/* Create a server on the current device. cfg may be NULL (width must be 4;
 * split_target, exit_fraction_pct and min_rounds are honoured). The number
 * of slots is min(max_slots, frontier_bytes / (48 * (4*split_target + 4)))
 * (split_target 0 means 256): each slot owns its frontier records.
 * Returns NULL on failure. */
bpida_server *bpida_server_create(const bpida_config *cfg, size_t frontier_bytes, int max_slots);
/* Queue one request: host_board points to one packed 15-puzzle word (host
 * memory, read before returning). Thread-safe, non-blocking. */
bpida_status bpida_server_submit(bpida_server *sv, const uint64_t *host_board, uint64_t req_id);
/* Move up to max finished results into out; returns how many. Non-blocking. */
int bpida_server_poll(bpida_server *sv, bpida_result *out, int max);
/* Requests submitted and not yet finished. */
int bpida_server_in_flight(bpida_server *sv);
void bpida_server_get_stats(bpida_server *sv, bpida_server_stats *out);
/* The clock used for submit_time_s / done_time_s (seconds, monotonic). */
double bpida_server_clock(void);
/* Time slice of a device step (default 2000 microseconds; 0 = none). When a
 * step has searched for this long it stops, and every iteration it did not
 * finish continues in the next step from its open nodes, so requests with
 * short iterations finish (and new ones are admitted) without waiting for
 * the longest iteration on the GPU. Results do not depend on it. Takes
 * effect from the next step. */
void bpida_server_set_time_slice(bpida_server *sv, int microseconds);
/* Stop the service (pending requests are dropped) and free it. */
void bpida_server_destroy(bpida_server *sv);

/* Statistics of the last solve call made by this host thread, complete once
 * that call's stream has been synchronised (the loop counts of a
 * graph-driven call are copied back at its end; they are zero if the
 * workspace it used has served a later call since). If timing is on before
 * a call (bpida_set_timing(1)), search kernel durations are recorded with
 * CUDA events on the launching stream (driver = 1 only). */
void bpida_set_timing(int on);
void bpida_get_stats(bpida_stats *out);
/* The search kernel launches of this host thread's last solve call, if it
 * ran the host-driven loop (driver = 1) with timing on: launch i took ms[i]
 * milliseconds (CUDA events on the launching stream) and popped nodes[i]
 * nodes. Writes the first min(count, cap) entries of each non-null array and
 * returns the count (0 after a graph-driven call or with timing off). For
 * turning a profiler's per-launch instruction count into instructions per
 * expansion; not part of Algorithm 1. */
int bpida_get_launch_log(double *ms, uint64_t *nodes, int cap);

/* Fused iterations (calls of at most 8 boards without a node budget search
 * several consecutive thresholds in one step): a step fuses the next
 * thresholds while the highest of them is predicted (x8 per threshold) to
 * expand at most `nodes` nodes, divided among the call's active boards.
 * All-solutions results do not depend on it; only the number of steps and
 * the nodes searched above a board's optimum do (first-solution mode: also
 * whether the final iteration's count is complete). 0 restores the default
 * (8e6). Process-wide; takes effect at the next call. */
void bpida_set_fuse_nodes(uint64_t nodes);

/* Free the calling device's workspaces (after waiting for their last calls)
 * and forget bpida_solve_noalloc's array address on it. */
void bpida_release_workspace(void);

/* ---- pattern-database heuristic ----
 * Additive disjoint pattern databases, the memory-intensive heuristic that
 * the paper's conclusion (Section 7) names as future work: kept in device
 * memory and read by the search kernels through L2.
 *
 * Tiles 1 .. W*W-1 are split into disjoint groups. For a group G with tiles
 * t_0 < ... < t_{k-1}, an abstract state is the positions of G's tiles and
 * of the blank; an abstract move swaps the blank with an adjacent cell and
 * costs 1 if that cell holds a tile of G, else 0. Table G holds, at index
 * sum_j pos(t_j) << 4j | blank << 4k (16^(k+1) bytes), the cost of a
 * cheapest abstract path to the abstract goal (tile t at cell t, blank at
 * 0), and 255 at indices that are no abstract state. h(board) = sum over
 * groups of the entry of the board's abstraction: admissible, consistent,
 * of the parity of the Manhattan distance and never below it, so every
 * convention above holds unchanged (limits still rise by exactly 2) and
 * results differ from the Manhattan ones only in the per-iteration node
 * counts, which are those of IDA* with this heuristic.
 */
typedef struct bpida_pdb bpida_pdb;

/* Builds the tables on the current device (on `stream`; returns once they
 * are built). width: 3 or 4. group_of_tile[t] (t = 1 .. W*W-1; entry 0 is
 * ignored) is t's group, numbered from 0 without gaps; at most 6 groups of
 * 1 to 6 tiles each (a 6-tile group's table is 256 MB). On success *out
 * owns the tables until bpida_pdb_destroy. Errors: BPIDA_EINVAL (bad
 * width or grouping), BPIDA_ENOMEM, BPIDA_ECUDA. */
bpida_status bpida_pdb_create(int width, const int *group_of_tile, bpida_pdb **out, void *stream);
/* Frees the tables (on the device they were built on), after waiting for the
 * device's work to finish (a solve call that reads them may still be
 * running on some stream). No call that uses `pdb` may be issued after. */
void bpida_pdb_destroy(bpida_pdb *pdb);
int bpida_pdb_groups(const bpida_pdb *pdb);
/* Bytes of group `group`'s table (0 for a bad group) and its largest entry
 * (-1 for a bad group). */
uint64_t bpida_pdb_table_bytes(const bpida_pdb *pdb, int group);
int bpida_pdb_max_value(const bpida_pdb *pdb, int group);
/* Copies group `group`'s table into dst (host or device memory, at least
 * bpida_pdb_table_bytes bytes) on `stream` and waits for the copy. */
bpida_status bpida_pdb_copy_table(const bpida_pdb *pdb, int group, uint8_t *dst, uint64_t bytes, void *stream);

/* bpida_solve_ex with the pattern-database heuristic `pdb` (built on the
 * current device, for cfg->width; width 0 means the tables' width).
 * cfg->variant must be 0 and cfg->stack_entries 0 (= 384), 384 or 512; everything
 * else (first-solution mode, node budgets, the graph and host drivers) is
 * as in bpida_solve_ex. Returns BPIDA_EINVAL for a null or foreign pdb. */
bpida_status bpida_solve_pdb(const bpida_config *cfg, const bpida_pdb *pdb, const uint64_t *boards, int n,
                             int *out_len, uint8_t *out_moves, uint64_t *out_nodes_per_iter,
                             int *out_num_iters, int *out_status, uint64_t *out_solutions, void *stream);

const char *bpida_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* BPIDA_H */
