// Device side of the GB300 Block-Parallel IDA* solver.
//
// Method (Horie & Fukunaga, "Block-Parallel IDA* for GPUs"):
//   * Algorithm 1, BPDFS: a group of threads shares one stack of open
//     nodes; each repetition pops several nodes at once, tests them for the
//     goal, generates children with f = g + cost + h, pushes those with
//     f <= limit (linearizable put) and keeps min f of the rest as f_next.
//     Here the group is one warp, one node per lane; children are pushed
//     with __ballot_sync/__popc slot reservation into a shared-memory ring.
//   * Algorithm 1, BPIDA*: a root set is built, the first limit is decided,
//     and each iteration searches every root's subtree in parallel. Here the
//     root set is rebuilt every iteration by k_split (a breadth-first,
//     order-preserving expansion of the top levels of the same depth-first
//     tree, without duplicate detection, so node counts stay those of
//     sequential IDA*), the first limit is h(start), and the next limit is
//     the smallest pruned f.
//   * Section 5's static load balancing (per-root work estimates from the
//     previous iteration) is replaced by a work queue consumed by persistent
//     warps plus hand-back: when enough warps have run dry, busy warps write
//     their open nodes back to a queue and the next pass redistributes them.
//
// Nothing in this file waits on another warp, block or kernel: every loop
// is bounded by the work it consumes, so no kernel can hang.
#pragma once
#include <stdint.h>
#include <limits.h>
#include <cuda_runtime.h>
#include <type_traits>

namespace bp {

typedef unsigned __int128 u128;

template <int W> struct Geo;
template <> struct Geo<3> {
    typedef uint64_t B;
    static constexpr int N = 9, BITS = 4, MAXLEN = 32, MAXIT = 17;
};
template <> struct Geo<4> {
    typedef uint64_t B;
    static constexpr int N = 16, BITS = 4, MAXLEN = 80, MAXIT = 41;
};
template <> struct Geo<5> {
    typedef u128 B;
    static constexpr int N = 25, BITS = 5, MAXLEN = 208, MAXIT = 105;
};

template <int W>
__host__ __device__ __forceinline__ typename Geo<W>::B goal_board()
{
    typedef typename Geo<W>::B B;
    B g = 0;
#pragma unroll
    for (int p = 0; p < Geo<W>::N; ++p)
        g |= (B)(unsigned)p << (Geo<W>::BITS * p);
    return g;
}

template <int W>
__host__ __device__ __forceinline__ unsigned tile_at(typename Geo<W>::B b, int p)
{
    return (unsigned)(b >> (Geo<W>::BITS * p)) & ((1u << Geo<W>::BITS) - 1u);
}

// ---- node metadata (32 bits) ----
//  bits  0..4   blank position
//  bits  5..7   last move (0..3), 4 = none
//  bits  8..15  slack = limit - g - h  (>= 0 for every stored node)
//  bits 16..20  records: depth below the split root; stack: origin slot
//  bit  21      records: goal found above the split depth (a leaf)
__host__ __device__ __forceinline__ uint32_t m_blank(uint32_t m) { return m & 31u; }
__host__ __device__ __forceinline__ uint32_t m_last(uint32_t m) { return (m >> 5) & 7u; }
__host__ __device__ __forceinline__ int m_slack(uint32_t m) { return (int)((m >> 8) & 255u); }
__host__ __device__ __forceinline__ uint32_t m_hi(uint32_t m) { return (m >> 16) & 31u; }
static constexpr uint32_t M_LEAF = 1u << 21;
static constexpr uint32_t M_NODE_MASK = 0xFFFFu;
static constexpr uint32_t LAST_NONE = 4u;
__host__ __device__ __forceinline__ uint32_t m_make(uint32_t blank, uint32_t last, uint32_t slack)
{
    return blank | (last << 5) | (slack << 8);
}

// A frontier / queue record.
template <int W> struct Rec {
    typename Geo<W>::B b;
    uint32_t meta;
    uint32_t inst;    // instance index
    uint32_t origin;  // index of the frontier record this node descends from
    uint32_t pm;      // moves from the split root, 2 bits each, first lowest
};

// ---- Manhattan move table ----
// For blank position p and move m, word e[p][m]:
//   bit 0        the move keeps the blank on the board
//   bit t (t>0)  sliding tile t from the blank's new position into p moves
//                it away from its goal cell (h rises by 1; else h falls by 1)
template <int W> struct MoveLut { uint32_t e[Geo<W>::N][4]; };

// Builds the table on the host (Manhattan distance of tile t from its goal
// cell before and after it slides into the blank).
template <int W> inline MoveLut<W> make_move_lut()
{
    MoveLut<W> L;
    for (int p = 0; p < Geo<W>::N; ++p)
        for (int m = 0; m < 4; ++m)
            L.e[p][m] = 0u;
    const int dr[4] = {-1, 0, 0, 1}, dc[4] = {0, -1, 1, 0};
    for (int p = 0; p < W * W; ++p) {
        const int r = p / W, c = p % W;
        for (int m = 0; m < 4; ++m) {
            const int rr = r + dr[m], cc = c + dc[m];
            if (rr < 0 || rr >= W || cc < 0 || cc >= W)
                continue;
            uint32_t e = 1u;
            for (int t = 1; t < W * W; ++t) {
                const int gr = t / W, gc = t % W;
                const int before = (rr > gr ? rr - gr : gr - rr) + (cc > gc ? cc - gc : gc - cc);
                const int after = (r > gr ? r - gr : gr - r) + (c > gc ? c - gc : gc - c);
                if (after > before)
                    e |= 1u << t;
            }
            L.e[p][m] = e;
        }
    }
    return L;
}

// Per-lane view of one table row. W <= 4: the four 16-bit masks of a row
// are packed into one 64-bit word, so a warp reads the 16 rows from 32
// distinct banks. W = 5: a 16-byte row, held as two arrays of 8-byte halves
// (words 0-1 of the 25 rows, then words 2-3): a half-warp's 8-byte loads of
// one array share a bank only for positions 16 apart (16-byte rows shared
// banks every 8 positions).
template <int W, bool Narrow = (W <= 4)> struct LutRow;
template <int W> struct LutRow<W, true> {
    uint64_t v;
    __device__ __forceinline__ bool legal(int m) const { return (v >> (16 * m)) & 1u; }
    __device__ __forceinline__ bool away(int m, unsigned t) const { return (v >> (16 * m + t)) & 1u; }
};
template <int W> struct LutRow<W, false> {
    uint4 v;
    __device__ __forceinline__ uint32_t w(int m) const { return m == 0 ? v.x : m == 1 ? v.y : m == 2 ? v.z : v.w; }
    __device__ __forceinline__ bool legal(int m) const { return w(m) & 1u; }
    __device__ __forceinline__ bool away(int m, unsigned t) const { return (w(m) >> t) & 1u; }
};

template <int W> struct SharedLut {
    static constexpr int BYTES = (W <= 4) ? 8 * 16 : 16 * 25;
    // fills shared memory from the kernel-parameter copy (block-wide)
    __device__ static void load(unsigned char *dst, const MoveLut<W> &src)
    {
        if (W <= 4) {
            uint64_t *d = (uint64_t *)dst;
            for (int p = threadIdx.x; p < Geo<W>::N; p += blockDim.x) {
                uint64_t v = 0;
                for (int m = 0; m < 4; ++m)
                    v |= (uint64_t)(src.e[p][m] & 0xFFFFu) << (16 * m);
                d[p] = v;
            }
        } else {
            // bits 28..31 of the first word: the four legal bits again (bit
            // 28 + m: move m), so that one shift gives the position's moves
            // (tiles are at most 24: the away bits stay below)
            uint2 *d = (uint2 *)dst;
            for (int p = threadIdx.x; p < Geo<W>::N; p += blockDim.x) {
                uint32_t legal = 0;
                for (int m = 0; m < 4; ++m)
                    legal |= (src.e[p][m] & 1u) << (28 + m);
                d[p] = make_uint2(src.e[p][0] | legal, src.e[p][1]);
                d[Geo<W>::N + p] = make_uint2(src.e[p][2], src.e[p][3]);
            }
        }
    }
    __device__ static __forceinline__ LutRow<W> row(const unsigned char *base, int p)
    {
        LutRow<W> r;
        if constexpr (W <= 4) {
            r.v = ((const uint64_t *)base)[p];
        } else {
            const uint2 lo = ((const uint2 *)base)[p], hi = ((const uint2 *)base)[Geo<W>::N + p];
            r.v = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
        return r;
    }
};

// Blank displacement of move m: up, left, right, down.
template <int W> __device__ __forceinline__ int move_off(int m)
{
    return m == 0 ? -W : m == 1 ? -1 : m == 2 ? 1 : W;
}

// ---- control block (device memory; the loop state of one solve call) ----
struct Ctrl {
    int n_in;         // records in this pass's input queue
    int head;         // next input record to take
    int out_count;    // records handed back during this pass
    int exited;       // warps that found the input exhausted
    int err;          // error bits (ERR_*)
    int n_active;     // problems in this step
    int n_next;       // problems for the next step
    int cur;          // which active list holds this step's problems
    int qi;           // which queue is this pass's input
    int steps;        // threshold steps completed
    int passes_step;  // search passes in this step
    int max_out;      // largest hand-back of one pass
    int pass_again;   // set at the end of a pass: another pass follows
    int step_again;   // set at the end of a step: another step follows
    int first_pass;   // 1: this pass reads the splitter's frontiers in place
    int done_warps;   // search blocks finished in this pass (one warp each in the paper kernel)
    int done_blocks;  // blocks finished in the current split / advance / init
    int n_front;      // records of this step's frontiers (the first pass's input starts with them)
    int n_carry;      // serving: open nodes carried over from the previous step
    int carry_q;      // serving: the queue that holds them
    unsigned long long step_t0;  // start of this step (%globaltimer)
    int n_done;       // serving: entries of the done list
    unsigned long long records_total;
    unsigned long long handed_back_total;
    unsigned long long search_nodes_total;  // nodes popped by k_search
    unsigned long long spills;              // stack overflows handed back
    unsigned long long passes_total;
    unsigned long long search_ns;           // sum of k_search durations (globaltimer)
    unsigned long long t_start, t_end;      // this pass's first block start / last block end
};
static constexpr int MAX_STEPS = 100000;        // loop guards: exceeding one is an
static constexpr int MAX_PASSES_PER_STEP = 100000;  // internal error, never a hang

// ---- one call's arguments (device memory, written before the loop) ----
struct CallDesc {
    const uint64_t *boards;
    int *out_len;
    uint8_t *out_moves;
    unsigned long long *out_nodes;
    int *out_iters;
    int *out_status;
    unsigned long long *out_solutions;  // may be null
    unsigned long long node_budget;
    int n;
    int first_only;  // 1: stop an instance's search at its first goal
};

static constexpr int ERR_QUEUE = 1;      // hand-back queue full
static constexpr int ERR_INTERNAL = 2;   // consistency check failed

// ---- per-instance state ----
enum { MODE_COUNT = 0, MODE_PATH = 1, MODE_DONE = 2 };
template <int W> struct InstState {
    typename Geo<W>::B start;
    typename Geo<W>::B root;     // root of the next split
    uint32_t start_meta;         // blank | none | 0
    uint32_t root_meta;          // blank | last | slack
    int h0;
    int limit;
    int it;                      // index of the current iteration
    int rows;                    // node-count rows written
    int path_len;
    int mode;
    int status;
    int length;
    uint32_t target;             // frontier records wanted from the next split
    int jump;                    // iterations fused above `limit` in the current step (see Fuse)
    unsigned long long cum_nodes;
    unsigned long long solutions;
};

struct Counters {
    unsigned long long *search_nodes;  // nodes popped inside the search kernel
    unsigned long long *split_nodes;   // nodes expanded by the splitter
    int *fnext_off;                    // min over pruned children of f - limit
    unsigned long long *goals;         // goal nodes popped
    unsigned *goal_origin;             // smallest origin of a goal-bearing record
    unsigned long long *budget_left;   // search nodes this iteration may pop (~0 = no budget)
    unsigned *aborted;                 // bit 0: the node budget ran out in this iteration;
                                       // bit 1: first-solution mode found a goal
};
static constexpr unsigned ABORT_BUDGET = 1u, ABORT_FOUND = 2u;

// Fused iterations. The Manhattan distance is consistent (h changes by
// exactly 1 per move), so f never decreases along a path, and sequential
// IDA* at limit L pops exactly the nodes with f <= L whose ancestors are not
// goals. One search at limit L + 2J therefore pops the nodes of the
// iterations L, L + 2, ..., L + 2J together; counting the popped nodes by
// slack (limit + 2J - f) gives each of those iterations' node count, and
// counting goals by slack gives the first limit with a solution, its number
// of optimal solutions and its first goal-bearing frontier record. A step
// fuses the iterations whose counts are predicted to stay small, so the
// results are exactly those of one iteration per step.
static constexpr int FUSE_MAX = 6;  // at most FUSE_MAX + 1 iterations per step
static constexpr int FUSE_K = 8;    // per-instance entries of the fused counters
struct Fuse {
    int *jump;                     // per instance: J of this step (null: no fusion)
    unsigned long long *low;       // per instance x FUSE_K: nodes popped (split and search) with slack 2m, m < J
    unsigned long long *goals;     // per instance x FUSE_K: goals popped with slack 2(J - j), by j
    unsigned *origin;              // per instance x FUSE_K: smallest origin of such a goal, by j
    unsigned long long max_nodes;  // fuse while the top iteration is predicted below this,
                                   // divided among the instances of the step (nodes that
                                   // overshoot the optimum cost every instance; the
                                   // steps saved are shared)
};

// Additive disjoint pattern databases: the memory-intensive heuristic that
// the paper's conclusion names as future work (Section 7), kept in global
// memory and read through L2. Tiles 1..N-1 are split into disjoint groups;
// group G's table holds, for every placement of its tiles and of the blank,
// the fewest moves of G's own tiles that bring G home (moves of other tiles
// are free), at index sum_j pos(t_j) << 4j | blank << 4k (t_0 < ... < t_{k-1}
// its tiles), and h is the sum over groups. A move changes one group's
// value by exactly 1 and no other (the blank's position is part of every
// entry), so h is consistent, has the parity of the Manhattan distance, and
// the search's slack arithmetic (a child keeps slack s or drops to s - 2) is
// the Manhattan one; only the direction of the step is read from a table.
//
// Tiles are renumbered into slots (slot 0: the blank; then the groups'
// tiles, group by group, in increasing order). The search kernel's stack
// entries (24 bytes) hold the slot board (4-bit field p: the slot of the
// tile at cell p) and the inverse board (field s: the cell of the tile in
// slot s), so the tile that moves is one field of the first, and a group's
// index is one field of the second plus the blank's nibble; the metadata
// carries h_g mod 4 of every group (enough to tell h_g + 1 from h_g - 1).
static constexpr int PDB_MAX_GROUPS = 6;
static constexpr int PDB_MAX_TILES = 6;    // per group: a table of 16^(k+1) bytes (256 MB at k = 6)
static constexpr int PDB_VSHIFT = 20;      // stack metadata: h_g mod 4 at bits 20 + 2g
static constexpr uint32_t PDB_VMASK = 0xFFF00000u;
struct PdbSlot {
    unsigned goff;  // bit offset of the slot's group field in the inverse board
    unsigned mask;  // (1 << field width) - 1
    unsigned vsh;   // metadata bit of h_g mod 4
    unsigned base;  // byte offset of the group's table
};
struct PdbInfo {
    PdbSlot slot[16];  // per slot s >= 1 (slot 0: zero)
    unsigned char slot_of_tile[16], tile_of_slot[16];
    int ng;
    int goff[PDB_MAX_GROUPS], gbits[PDB_MAX_GROUPS];
    unsigned base[PDB_MAX_GROUPS];
};
struct PdbDev {
    const unsigned char *tab;  // all groups' tables, one after another (null: Manhattan distance)
    const PdbInfo *info;       // device copy of the layout
    unsigned long long goal;   // the goal's inverse board
    unsigned long long goal_sb;  // the goal's slot board
};

struct Tune {
    int min_rounds;      // rounds before a warp may hand its stack back
    int exit_threshold;  // warps that must have run dry first
    int nodes_per_record;
    int target_cap;      // per-problem frontier cap
    int target_path;     // frontier records wanted for a path step
    int growth;          // expected node growth per iteration (x)
    int min_pass_ns;     // a pass hands work back only after running this long
    unsigned long long step_ns;  // serving: time slice of a step (0 = none)
};

// ---------------------------------------------------------------------
// Warp-level helpers
// ---------------------------------------------------------------------
static constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int warp_min_int(int v)
{
#pragma unroll
    for (int d = 16; d; d >>= 1)
        v = min(v, __shfl_xor_sync(FULL, v, d));
    return v;
}
__device__ __forceinline__ unsigned warp_min_u32(unsigned v)
{
#pragma unroll
    for (int d = 16; d; d >>= 1)
        v = min(v, __shfl_xor_sync(FULL, v, d));
    return v;
}

// Block-wide exclusive scan of small non-negative ints (blockDim <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(FULL, x, d);
        if (lane >= d)
            x += y;
    }
    if (lane == 31)
        warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(FULL, s, d);
            if (lane >= d)
                s += y;
        }
        if (lane < nw)
            warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    int before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before;
}

// ---------------------------------------------------------------------
// Device view of one solve call's workspace, passed to every kernel.
// ---------------------------------------------------------------------
template <int W> struct Dev {
    Ctrl *ctrl;
    const CallDesc *desc;
    InstState<W> *state;
    unsigned *act0, *act1;      // active problem lists (ctrl->cur selects)
    Rec<W> *scratch;            // per problem: 2 * C records
    Rec<W> *q0, *q1;            // pass queues (ctrl->qi selects the input)
    int *count, *offset;        // per problem: final-level records, prefix
    int C;
    int Q;                      // capacity of each queue
    Counters cnt;
    Tune tune;
    MoveLut<W> lut;
    cudaGraphConditionalHandle h_step, h_pass;
    int graph;                  // 1 inside the CUDA graph (sets the loop conditions)
    unsigned *done_list;        // serving: instances that finished in this step (else null)
    unsigned char *ovf;         // per-warp overflow stacks in global memory (may be null)
    int ovf_cap;                // entries per warp overflow stack (0 = none)
    Fuse fuse;                  // fused iterations (fuse.jump null: one iteration per step)
    // Serving with time slices (slice = 1): an instance's iteration may run
    // over several steps. Frontier regions then belong to instance slots, not
    // to positions in the active list; carry[i] = 1 marks a slot whose open
    // nodes were carried into the next step (no split, no advance), and
    // fbase[i] / fcount[i] locate the frontier of its current iteration.
    int slice;
    unsigned *carry;
    int *fbase, *fcount;
    PdbDev pdb;                 // pattern databases (solve calls with a PDB heuristic)
};

__device__ __forceinline__ unsigned long long global_ns();

// Frontier region of the problem at active position k (instance inst).
template <int W> __device__ __forceinline__ size_t region_of(const Dev<W> &a, int k, unsigned inst)
{
    return (size_t)(a.slice ? (int)inst : k) * 2 * (size_t)a.C;
}

// The step's time slice is over (serving).
template <int W> __device__ __forceinline__ bool slice_over(const Dev<W> &a)
{
    return a.slice && a.tune.step_ns &&
           global_ns() - *(volatile unsigned long long *)&a.ctrl->step_t0 > a.tune.step_ns;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- pattern-database helpers ----
// Copies the layout into shared memory (block-wide; a barrier follows).
__device__ __forceinline__ void pdb_load_info(PdbInfo *dst, const PdbInfo *src)
{
    for (int i = threadIdx.x; i < (int)(sizeof(PdbInfo) / 4); i += blockDim.x)
        ((unsigned *)dst)[i] = ((const unsigned *)src)[i];
}
// The inverse board of a position -> tile board.
template <int W> __device__ __forceinline__ uint64_t pdb_inverse(uint64_t b, const PdbInfo &pi)
{
    uint64_t v = 0;
#pragma unroll
    for (int p = 0; p < Geo<W>::N; ++p)
        v |= (uint64_t)p << (4 * pi.slot_of_tile[tile_at<W>(b, p)]);
    return v;
}
// A search stack board: inverse board (high half) and slot board (low half).
template <int W> __device__ __forceinline__ u128 pdb_encode(uint64_t b, const PdbInfo &pi)
{
    uint64_t inv = 0, sb = 0;
#pragma unroll
    for (int p = 0; p < Geo<W>::N; ++p) {
        const uint64_t s = pi.slot_of_tile[tile_at<W>(b, p)];
        inv |= (uint64_t)p << (4 * s);
        sb |= s << (4 * p);
    }
    return ((u128)inv << 64) | sb;
}
// The position -> tile board of an inverse board.
template <int W> __device__ __forceinline__ uint64_t pdb_board(uint64_t inv, const PdbInfo &pi)
{
    uint64_t b = 0;
#pragma unroll
    for (int s = 0; s < Geo<W>::N; ++s)
        b |= (uint64_t)pi.tile_of_slot[s] << (4 * ((inv >> (4 * s)) & 15u));
    return b;
}
// Table index of the group whose tiles sit in field [goff, goff + gbits).
__device__ __forceinline__ uint32_t pdb_index(uint64_t inv, uint32_t goff, uint32_t gbits)
{
    return ((uint32_t)(inv >> goff) & ((1u << gbits) - 1u)) | (((uint32_t)inv & 15u) << gbits);
}
// h of an inverse board (vb: h_g mod 4 of every group, as in the stack metadata).
__device__ __forceinline__ int pdb_h(const PdbDev &d, const PdbInfo &pi, uint64_t inv, uint32_t *vb)
{
    int h = 0;
    uint32_t bits = 0;
    for (int g = 0; g < pi.ng; ++g) {
        const uint32_t v = d.tab[pi.base[g] + pdb_index(inv, (uint32_t)pi.goff[g], (uint32_t)pi.gbits[g])];
        h += (int)v;
        bits |= (v & 3u) << (PDB_VSHIFT + 2 * g);
    }
    if (vb)
        *vb = bits;
    return h;
}
// For each move m whose bit is set in legal: whether sliding the tile at
// np[m] into the blank at p raises h (bit m of the result; else h falls by
// 1); inv is the parent's inverse board. The eight table reads (the moved
// tile's group entry of child and parent, per move) are issued before any
// of them is used, so that their latencies overlap.
__device__ __forceinline__ unsigned pdb_away4(const PdbDev &d, const PdbInfo &pi, uint64_t inv, uint32_t p,
                                              const uint32_t np[4], const unsigned tile[4], unsigned legal)
{
    unsigned vc[4], vp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        vc[m] = vp[m] = 0;
        if ((legal >> m) & 1u) {
            const uint32_t j = pi.slot_of_tile[tile[m]];
            const PdbSlot sl = pi.slot[j];
            const uint64_t dd = (uint64_t)(p ^ np[m]);
            const uint64_t child = inv ^ (dd << (4 * j)) ^ dd;
            const unsigned char *t = d.tab + sl.base;
            const uint32_t gbits = (uint32_t)__popc(sl.mask);
            vc[m] = t[pdb_index(child, sl.goff, gbits)];
            vp[m] = t[pdb_index(inv, sl.goff, gbits)];
        }
    }
    unsigned away = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        away |= (vc[m] > vp[m] ? 1u : 0u) << m;
    return away;
}

// ---- warp stack entries ----
// Stack metadata (32 bits), different from the record metadata:
//  bits 0..6   BITS * blank position (the blank's field offset in the board)
//  bits 7..10  excluded move mask (the inverse of the move that made the
//              node; 0 for an instance root)
//  bits 11..18 slack = limit - g - h
template <int W> __device__ __forceinline__ uint32_t sm_from_rec(uint32_t m)
{
    const uint32_t last = m_last(m);
    const uint32_t excl = last < 4u ? (1u << (3u - last)) : 0u;
    return (m_blank(m) * (uint32_t)Geo<W>::BITS) | (excl << 7) | ((uint32_t)m_slack(m) << 11);
}
template <int W> __device__ __forceinline__ uint32_t rec_from_sm(uint32_t m)
{
    const uint32_t excl = (m >> 7) & 15u;
    const uint32_t last = excl ? 3u - (uint32_t)(__ffs(excl) - 1) : LAST_NONE;
    return m_make((m & 127u) / (uint32_t)Geo<W>::BITS, last, (m >> 11) & 255u);
}

// ---- the 15-puzzle search step, four moves at once ----
// With the Manhattan distance on the 4x4 board, the four candidate moves of
// a node are handled together: their neighbour tiles are gathered into the
// four bytes of one word (byte m: move m, in the order up, left, right,
// down), and whether each tile slides away from its goal cell is one packed
// comparison against per-position thresholds:
//   up    (tile from row r-1 to r): away iff t < 4r
//   left  (tile from col c-1 to c): away iff (t & 3) < c
//   right (tile from col c+1 to c): away iff 3 - (t & 3) < 3 - c
//   down  (tile from row r+1 to r): away iff 15 - t < 12 - 4r
// Each byte holds x = the tile term (at most 15) and the per-position table
// holds a + 127 (a = the threshold, at most 15), so (a + 127 - x) sets bit 7
// of its byte exactly when x < a and never borrows from the next byte.
// The search stack's metadata for this step sets bit 8m + 7 when move m is
// the inverse of the parent's move (it is excluded), keeps the blank's
// position in bits 0..3 and the slack in bits 8..14 (slack <= 80: the
// longest limit).
template <int W, bool PDB> struct FourMoves {
    static constexpr bool on = W == 4 && !PDB;
};
static constexpr uint32_t FM_BIT7 = 0x80808080u;
__device__ __forceinline__ uint32_t fm_from_rec(uint32_t m)
{
    const uint32_t last = m_last(m);
    const uint32_t excl = last < 4u ? (0x80u << (8u * (3u - last))) : 0u;
    return m_blank(m) | ((uint32_t)m_slack(m) << 8) | excl;
}
__device__ __forceinline__ uint32_t rec_from_fm(uint32_t m)
{
    const uint32_t e = m & FM_BIT7;
    const uint32_t last = e ? 3u - (uint32_t)((__ffs((int)e) - 1) >> 3) : LAST_NONE;
    return m_make(m & 15u, last, (m >> 8) & 127u);
}
// Per blank position p, in shared memory, six arrays of 16 eight-byte
// entries (a half-warp reads any 16 entries of one array without a bank
// conflict):
//   [p]      x: byte selector of the neighbours (up, left, right, down) in
//               the board viewed as 8 bytes (an off-board neighbour selects
//               byte 0); y: 0x0F in byte m when neighbour m's tile is the
//               low nibble of its byte
//   [16 + p] x: per byte m, 127 + the threshold of move m; y: bit 8m + 7 set
//               when move m keeps the blank on the board
//   [32 + p], [48 + p], [64 + p], [80 + p]: per move m, the low (moves 0-1,
//               2-3) and high (moves 0-1, 2-3) 32-bit words of 16^p +
//               16^(p + displacement of m) (0 for a move off the board).
struct FourMoveTable {
    static constexpr int BYTES = 16 * 16 + 16 * 32;
    __device__ static void load(uint2 *t)
    {
        for (int p = threadIdx.x; p < 16; p += blockDim.x) {
            const int r = p >> 2, c = p & 3;
            const int np[4] = {p - 4, p - 1, p + 1, p + 4};
            const bool on[4] = {r > 0, c > 0, c < 3, r < 3};
            const int thr[4] = {4 * r, c, 3 - c, 12 - 4 * r};
            uint32_t sel = 0, lowm = 0, z = 0, legal = 0;
            for (int m = 0; m < 4; ++m) {
                const int q = on[m] ? np[m] : 0;
                sel |= (uint32_t)(q >> 1) << (4 * m);
                if ((q & 1) == 0)
                    lowm |= 0x0Fu << (8 * m);
                z |= (uint32_t)(127 + thr[m]) << (8 * m);
                if (on[m])
                    legal |= 0x80u << (8 * m);
            }
            // per 32-bit half: 16^p for the blank's field (it gets the tile)
            // less 16^np for the neighbour's (it loses it), modulo 2^32
            uint32_t lo[4], hi[4];
            for (int m = 0; m < 4; ++m) {
                lo[m] = hi[m] = 0u;
                if (!on[m])
                    continue;
                const int q[2] = {p, np[m]};
                for (int k = 0; k < 2; ++k) {
                    const uint32_t f = 1u << (4 * (q[k] & 7));
                    uint32_t &h = q[k] < 8 ? lo[m] : hi[m];
                    h = k == 0 ? h + f : h - f;
                }
            }
            t[p] = make_uint2(sel, lowm);
            t[16 + p] = make_uint2(z, legal);
            t[32 + p] = make_uint2(lo[0], lo[1]);
            t[48 + p] = make_uint2(lo[2], lo[3]);
            t[64 + p] = make_uint2(hi[0], hi[1]);
            t[80 + p] = make_uint2(hi[2], hi[3]);
        }
    }
};
// ---- the 24-puzzle search step in the blank's frame ----
// The 24-puzzle's search stacks hold each board turned so that the blank is
// in field 0: field j holds the tile of cell (p + j) mod 25, p the blank's
// cell (the 125 used bits rotated right by 5p). The four neighbours then sit
// in fixed fields (up 20, left 24, right 1, down 5), and sliding the tile t
// of field j into the blank gives the child in its own blank's frame as the
// parent turned by a fixed amount:
//   child = rotr(R, 5j) ^ t ^ (t << 5(25 - j))
// (field 0 turns from t to the blank; field 25 - j, the parent's blank cell,
// gets t). Every shift has a constant amount, where the board's own frame
// needs a 128-bit shift by the blank's position per tile read and per child.
// Records (queues, frontiers) keep the board's own frame; the stack entry's
// metadata is the same in both.
template <int W, bool PDB> struct BlankFrame {
    static constexpr bool on = W == 5 && !PDB;
};
static constexpr u128 BOARD125 = (((u128)1) << 125) - 1u;
// sh = 5p, the blank's field offset (0 <= sh < 125)
__device__ __forceinline__ u128 to_blank_frame(u128 b, uint32_t sh)
{
    return sh ? (((b >> sh) | (b << (125u - sh))) & BOARD125) : b;
}
__device__ __forceinline__ u128 from_blank_frame(u128 r, uint32_t sh)
{
    return sh ? (((r << sh) | (r >> (125u - sh))) & BOARD125) : r;
}

// Shared memory of the search kernel before the warp stacks.
template <int W, bool PDB = false> struct SearchSmem {
    static constexpr int TABLES = SharedLut<W>::BYTES + (FourMoves<W, PDB>::on ? FourMoveTable::BYTES : 0);
};

// W <= 4: one 16-byte entry {board lo, board hi, meta, origin}.
// W == 5, and the pattern-database search: a 16-byte board array (the
// 128-bit board; slot board and inverse board) and an 8-byte {meta, origin}
// array.
template <int W, bool Wide = (W == 5)> struct WarpStack;
template <int W> struct WarpStack<W, false> {
    typedef uint64_t Board;
    static constexpr int ENTRY_BYTES = 16;
    uint4 *e;
    __device__ __forceinline__ void init(unsigned char *base, int) { e = (uint4 *)base; }
    __device__ __forceinline__ void put(int i, uint64_t b, uint32_t meta, uint32_t org)
    {
        e[i] = make_uint4((uint32_t)b, (uint32_t)(b >> 32), meta, org);
    }

    __device__ __forceinline__ void get(int i, uint64_t &b, uint32_t &meta, uint32_t &org) const
    {
        const uint4 v = e[i];
        b = ((uint64_t)v.y << 32) | v.x;
        meta = v.z;
        org = v.w;
    }
};
template <int W> struct WarpStack<W, true> {
    typedef u128 Board;
    static constexpr int ENTRY_BYTES = 24;
    uint4 *eb;
    uint2 *em;
    __device__ __forceinline__ void init(unsigned char *base, int S)
    {
        eb = (uint4 *)base;
        em = (uint2 *)(eb + S);
    }
    __device__ __forceinline__ void put(int i, u128 b, uint32_t meta, uint32_t org)
    {
        eb[i] = make_uint4((uint32_t)b, (uint32_t)(b >> 32), (uint32_t)(b >> 64), (uint32_t)(b >> 96));
        em[i] = make_uint2(meta, org);
    }
    __device__ __forceinline__ void get(int i, u128 &b, uint32_t &meta, uint32_t &org) const
    {
        const uint4 v = eb[i];
        b = ((u128)v.w << 96) | ((u128)v.z << 64) | ((u128)v.y << 32) | v.x;
        const uint2 m = em[i];
        meta = m.x;
        org = m.y;
    }
};

// The search stack of k_search's Manhattan step (15-puzzle four-move step,
// 24-puzzle in the blank's frame), with the layouts of WarpStack<W, false>
// and WarpStack<W, true>, addressed through the 32-bit shared window with
// explicit ld.shared/st.shared. A child is pushed by one predicated store
// (put_if) and the slot (15-puzzle: the slot's shared-window address)
// advances by the predicate, so the four moves of a node run without a
// branch around each push. (This stack lives in shared memory only: the
// global-memory overflow stacks keep WarpStack.)
template <bool Wide> struct SharedStack;
template <> struct SharedStack<false> {
    typedef uint64_t Board;
    static constexpr int ENTRY_BYTES = 16;
    uint32_t e;  // shared-window address of entry 0
    __device__ __forceinline__ void init(unsigned char *base, int) { e = (uint32_t)__cvta_generic_to_shared(base); }
    // shared-window address of entry i
    __device__ __forceinline__ uint32_t addr(int i) const { return e + 16u * (uint32_t)i; }
    // stores the entry at shared-window address a if p is nonzero
    __device__ __forceinline__ void put_if(uint32_t p, uint32_t a, uint64_t b, uint32_t meta, uint32_t org)
    {
        asm volatile("{ .reg .pred q; setp.ne.u32 q, %0, 0; @q st.shared.v4.u32 [%1], {%2, %3, %4, %5}; }"
                     :: "r"(p), "r"(a), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)), "r"(meta), "r"(org) : "memory");
    }
    __device__ __forceinline__ void put(int i, uint64_t b, uint32_t meta, uint32_t org)
    {
        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                     :: "r"(e + 16u * (uint32_t)i), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)), "r"(meta), "r"(org)
                     : "memory");
    }
    __device__ __forceinline__ void get(int i, uint64_t &b, uint32_t &meta, uint32_t &org) const
    {
        uint32_t x, y;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x), "=r"(y), "=r"(meta), "=r"(org) : "r"(e + 16u * (uint32_t)i) : "memory");
        b = ((uint64_t)y << 32) | x;
    }
};
template <> struct SharedStack<true> {
    typedef u128 Board;
    static constexpr int ENTRY_BYTES = 24;
    uint32_t eb, em;  // shared-window addresses of board 0 and {meta, origin} 0
    __device__ __forceinline__ void init(unsigned char *base, int S)
    {
        eb = (uint32_t)__cvta_generic_to_shared(base);
        em = eb + 16u * (uint32_t)S;
    }
    // stores entry i if p is nonzero
    __device__ __forceinline__ void put_if(uint32_t p, int i, u128 b, uint32_t meta, uint32_t org)
    {
        asm volatile("{ .reg .pred q; setp.ne.u32 q, %0, 0; @q st.shared.v4.u32 [%1], {%2, %3, %4, %5}; "
                     "@q st.shared.v2.u32 [%6], {%7, %8}; }"
                     :: "r"(p), "r"(eb + 16u * (uint32_t)i), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)),
                        "r"((uint32_t)(b >> 64)), "r"((uint32_t)(b >> 96)), "r"(em + 8u * (uint32_t)i), "r"(meta),
                        "r"(org) : "memory");
    }
    __device__ __forceinline__ void put(int i, u128 b, uint32_t meta, uint32_t org) { put_if(1u, i, b, meta, org); }
    __device__ __forceinline__ void get(int i, u128 &b, uint32_t &meta, uint32_t &org) const
    {
        uint32_t x, y, z, w;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(eb + 16u * (uint32_t)i) : "memory");
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(meta), "=r"(org) : "r"(em + 8u * (uint32_t)i) : "memory");
        b = ((u128)w << 96) | ((u128)z << 64) | ((u128)y << 32) | x;
    }
};

// Legal blank moves of every position as one integer constant: the 4-bit
// mask of position p (bit m = move m keeps the blank on the board) sits at
// bit BITS*p, so the blank's field offset indexes it directly.
template <int W> struct LegalMoves {
    typedef typename std::conditional<(W <= 4), uint64_t, u128>::type T;
    __host__ __device__ static constexpr T make()
    {
        T v = 0;
        for (int p = 0; p < W * W; ++p) {
            const int r = p / W, c = p % W;
            const unsigned m = (r > 0 ? 1u : 0u) | (c > 0 ? 2u : 0u) | (c < W - 1 ? 4u : 0u) | (r < W - 1 ? 8u : 0u);
            v |= (T)m << (Geo<W>::BITS * p);
        }
        return v;
    }
    __device__ static __forceinline__ unsigned at_sh(uint32_t sh)
    {
        constexpr T V = make();
        return (unsigned)(V >> sh) & 15u;
    }
};

// Field access by bit offset. For 64-bit boards the PTX shifts are used
// because PTX defines out-of-range amounts (clamped to 64): the offset of an
// illegal move then yields tile 0 / an unchanged board and needs no select.
template <int W, bool Wide = (W == 5)> struct BoardOps;
template <int W> struct BoardOps<W, false> {
    __device__ static __forceinline__ unsigned tile(uint64_t b, uint32_t sh)
    {
        uint64_t r;
        asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(b), "r"(sh));
        return (unsigned)r & 15u;
    }
    __device__ static __forceinline__ uint64_t flip(uint64_t b, uint32_t v, uint32_t sh)
    {
        uint64_t x;
        asm("shl.b64 %0, %1, %2;" : "=l"(x) : "l"((uint64_t)v), "r"(sh));
        return b ^ x;
    }
};
template <int W> struct BoardOps<W, true> {
    __device__ static __forceinline__ unsigned tile(u128 b, uint32_t sh)
    {
        return sh < 128u ? ((unsigned)(b >> sh) & 31u) : 0u;
    }
    __device__ static __forceinline__ u128 flip(u128 b, uint32_t v, uint32_t sh)
    {
        return sh < 128u ? (b ^ ((u128)v << sh)) : b;
    }
};

// Move tables for the XOR child update: sliding tile t between positions
// q = min(p, np) and q + |off| flips t in both fields, i.e.
// child = board ^ ((t * (1 + 2^(BITS*|off|))) << (BITS*q)).
template <int W> __device__ __forceinline__ unsigned move_mul(int m)
{
    constexpr int BITS = Geo<W>::BITS;
    return (m == 0 || m == 3) ? (1u + (1u << (BITS * W))) : (1u + (1u << BITS));
}

// away bit of the Manhattan table row for move m and tile t
template <int W> __device__ __forceinline__ bool away_bit(const LutRow<W> &row, int m, unsigned t)
{
    if constexpr (W <= 4) {
        const uint32_t lo = (uint32_t)row.v, hi = (uint32_t)(row.v >> 32);
        const uint32_t w = (m < 2) ? lo : hi;
        return (w >> (((m & 1) << 4) + t)) & 1u;
    } else {
        return (row.w(m) >> t) & 1u;
    }
}

template <int W> __device__ __forceinline__ LutRow<W> lut_row_sh(const unsigned char *base, uint32_t sh)
{
    return SharedLut<W>::row(base, (int)(sh / (uint32_t)Geo<W>::BITS));
}

// PDB: stack entries hold inverse boards; records hold boards.
template <int W, int S, bool PDB = false, typename Stack = WarpStack<W>>
__device__ __forceinline__ void hand_back_stack(const Dev<W> &a, Rec<W> *out, const Stack &stk,
                                                int from, int k, unsigned inst, int lane,
                                                const PdbInfo *pi = nullptr, bool fm = false, bool bf = false)
{
    if (k <= 0)
        return;
    int base = 0;
    if (lane == 0)
        base = atomicAdd(&a.ctrl->out_count, k);
    base = __shfl_sync(FULL, base, 0);
    if (base + k > a.Q) {
        if (lane == 0)
            atomicOr(&a.ctrl->err, ERR_QUEUE);
        return;
    }
    for (int j = lane; j < k; j += 32) {
        typename Stack::Board b;
        uint32_t m, o;
        stk.get(from + j, b, m, o);
        Rec<W> r;
        if constexpr (PDB)
            r.b = pdb_board<W>((uint64_t)(b >> 64), *pi);
        else if constexpr (W == 5)
            r.b = bf ? from_blank_frame(b, m & 127u) : b;
        else
            r.b = b;
        r.meta = fm ? rec_from_fm(m) : rec_from_sm<W>(m);
        r.inst = inst;
        r.origin = o;
        r.pm = 0;
        out[base + j] = r;
    }
}

// Input record idx of a pass. The first pass of a step reads the splitter's
// per-problem frontiers in place: problem k owns indices
// [offset[k], offset[k] + count[k]); the origin of a frontier record is its
// index. Later passes read the hand-back queue.
// Input record idx of a pass. The first pass of a step reads the frontiers
// in place (indices below n_front; problem k owns [offset[k], offset[k] +
// count[k]), and a frontier record's origin is its index), then the open
// nodes carried over from the previous step (serving), which sit in `in`.
// Later passes read the hand-back queue `in`.
template <int W>
__device__ __forceinline__ Rec<W> load_rec(const Dev<W> &a, bool frontier, int n_active, int n_front,
                                           const unsigned *act, const Rec<W> *in, int idx)
{
    if (!frontier)
        return in[idx];
    if (idx >= n_front)
        return in[idx - n_front];
    int lo = 0, hi = n_active - 1;  // last k with offset[k] <= idx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.offset[mid] <= idx)
            lo = mid;
        else
            hi = mid - 1;
    }
    Rec<W> r = a.scratch[region_of(a, lo, a.slice ? act[lo] : 0u) + (idx - a.offset[lo])];
    r.origin = (uint32_t)idx;
    return r;
}

template <int W>
__device__ __forceinline__ void hand_back_records(const Dev<W> &a, bool frontier, int n_active, int n_front,
                                                  const unsigned *act, const Rec<W> *in, Rec<W> *out, int from,
                                                  int to, int lane)
{
    const int k = to - from;
    if (k <= 0)
        return;
    int base = 0;
    if (lane == 0)
        base = atomicAdd(&a.ctrl->out_count, k);
    base = __shfl_sync(FULL, base, 0);
    if (base + k > a.Q) {
        if (lane == 0)
            atomicOr(&a.ctrl->err, ERR_QUEUE);
        return;
    }
    for (int j = lane; j < k; j += 32)
        out[base + j] = load_rec<W>(a, frontier, n_active, n_front, act, in, from + j);
}

template <int W> __device__ void end_of_pass(const Dev<W> &a);

// The search kernel's board type and its goal (PDB: inverse and slot
// boards in one 128-bit value).
template <int W, bool PDB> using SearchBoard = typename std::conditional<PDB, u128, typename Geo<W>::B>::type;
template <int W, bool PDB>
__device__ __forceinline__ SearchBoard<W, PDB> search_goal(const Dev<W> &a)
{
    if constexpr (PDB)
        return ((u128)a.pdb.goal << 64) | a.pdb.goal_sb;
    else
        return goal_board<W>();
}

// One warp = one shared stack (Algorithm 1's openList). Each round pops up
// to 32 nodes (one per lane), tests them for the goal, and generates the
// children of the rest; children with f <= limit are pushed at slots
// reserved by ballot/popc (a linearizable put with one writer per slot),
// the others only contribute f_next. The warp takes runs of same-instance
// records from the pass's input queue until it is exhausted; once enough
// warps have run dry, busy warps hand their open nodes to the next pass.
// FUSE: the kernel also counts popped nodes and goals by slack for fused
// iterations (see Fuse); without it that code is compiled out.
// PDB: the heuristic is the pattern databases' sum (stack entries hold
// inverse boards and h_g mod 4; see PdbInfo), else the Manhattan distance.
template <int W, int S, bool FUSE = false, bool PDB = false>
__global__ void k_search(const Dev<W> a)
{
    typedef typename Geo<W>::B B;
    typedef SearchBoard<W, PDB> SB;  // what a stack entry holds (B, or the PDB pair)
    constexpr int BITS = Geo<W>::BITS;
    constexpr bool FM = FourMoves<W, PDB>::on;           // four moves at once (15-puzzle)
    constexpr bool BF = BlankFrame<W, PDB>::on;          // boards in the blank's frame (24-puzzle)
    typedef WarpStack<W, (W == 5) || PDB> GStack;        // layout of the overflow stacks (global memory)
    typedef typename std::conditional<FM || BF, SharedStack<(W == 5) || PDB>, GStack>::type Stack;
    extern __shared__ __align__(16) unsigned char smem[];
    // end-of-pass bookkeeping is combined per block, so that the grid-wide
    // counters see one atomic per block instead of one per warp
    __shared__ int s_warps_done;
    __shared__ unsigned long long s_t_end, s_nodes;
    __shared__ unsigned s_low[FUSE ? 32 : 1][FUSE_MAX];  // fused iterations: per warp, pops with slack 2m
    unsigned char *lut = smem;
    if (threadIdx.x == 0) {
        atomicMin(&a.ctrl->t_start, global_ns());
        s_warps_done = 0;
        s_t_end = 0;
        s_nodes = 0;
    }
    SharedLut<W>::load(lut, a.lut);
    if constexpr (FourMoves<W, PDB>::on)
        FourMoveTable::load((uint2 *)(smem + SharedLut<W>::BYTES));
    const PdbInfo *pi = nullptr;
    if constexpr (PDB) {
        static_assert(W <= 4, "pattern databases: 8- and 15-puzzle");
        __shared__ PdbInfo s_pi;
        pdb_load_info(&s_pi, a.pdb.info);
        pi = &s_pi;
    }
    __syncthreads();
    const Rec<W> *in = a.ctrl->qi ? a.q1 : a.q0;
    Rec<W> *out = a.ctrl->qi ? a.q0 : a.q1;
    const bool frontier = a.ctrl->first_pass != 0;
    const int n_act = a.ctrl->n_active;
    const int n_front = a.ctrl->n_front;
    const unsigned *act = a.ctrl->cur ? a.act1 : a.act0;
    const bool first_only = a.desc->first_only != 0;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Stack stk;
    stk.init(smem + SearchSmem<W, PDB>::TABLES + (size_t)warp * S * Stack::ENTRY_BYTES, S);
    const uint2 *fmtab = (const uint2 *)(smem + SharedLut<W>::BYTES);
    // byte selectors and the slack step of the four-move children, read
    // from shared memory so that they stay multiplier operands
    __shared__ uint32_t s_one;
    if (threadIdx.x == 0)
        s_one = 1u;
    __syncthreads();
    const uint32_t one = *(volatile uint32_t *)&s_one;
    const uint32_t ebyte[4] = {one, one << 8, one << 16, one << 24};
    // signed byte 4 in byte m: with the away bits (0x80, i.e. -128 as a
    // signed byte) a signed dot product gives -512, the slack step of 2
    const int e4[4] = {(int)(4u * one), (int)((4u * one) << 8), (int)((4u * one) << 16), (int)((4u * one) << 24)};
    // this warp's overflow stack in global memory: the oldest open nodes go
    // there when the shared stack is full and come back when it drains
    // (24-puzzle only: its deeper trees overflow the shared stack often)
    constexpr bool OVF = (W == 5);
    GStack ovf;
    const size_t gwarp = (size_t)blockIdx.x * (blockDim.x >> 5) + warp;
    ovf.init(a.ovf + gwarp * (size_t)a.ovf_cap * GStack::ENTRY_BYTES, a.ovf_cap);
    int ovf_n = 0;
    const unsigned lt = (1u << lane) - 1u;
    const SB GOAL = search_goal<W, PDB>(a);
    const int n_in = a.ctrl->n_in;
    const int total_warps = gridDim.x * (blockDim.x >> 5);
    const int chunk = max(1, min(32, n_in / (total_warps * 4)));
    int rounds = 0;
    bool stop = false;
    // Node and pruned-f counters are accumulated per warp while its runs
    // belong to one instance and published when the instance changes, when
    // an instance has a node budget (its count gates the budget), and at the
    // end: fmin is this lane's smallest pruned f - limit for acc_inst.
    unsigned acc_inst = 0xffffffffu;
    unsigned long long acc_nodes = 0, tot_nodes = 0;
    int fmin = INT_MAX;
    // four-move step: bit 7 of a byte is set once a child was pruned; the
    // slack is even (f keeps the parity of h(start), and limits rise by 2),
    // so a node with slack < 2 has slack 0 and its pruned children f = limit + 2
    uint32_t prn = 0;
    // fused iterations: nodes popped with slack 2m (m < acc_J) of acc_inst,
    // counted by lane 0 in shared memory
    int acc_J = 0;
    unsigned *lowc = s_low[FUSE ? warp : 0];
    if (FUSE && lane == 0)
        for (int m = 0; m < FUSE_MAX; ++m)
            lowc[m] = 0;
    // per lane, between flushes into lowc (every 32 rounds and at the end of
    // a run): byte m counts this lane's pops with slack 2m, m < J (at most 32
    // per byte between flushes)
    unsigned long long lowp = 0;
    auto flush_low = [&](int J) {
        for (int m = 0; m < J; ++m) {
            const unsigned c = __reduce_add_sync(FULL, (unsigned)(lowp >> (8 * m)) & 255u);
            if (lane == 0)
                lowc[m] += c;
        }
        lowp = 0;
    };
    auto publish = [&]() {
        if (FM && prn)
            fmin = min(fmin, 2);
        prn = 0;
        const int fm = warp_min_int(fmin);
        if (lane == 0 && acc_inst != 0xffffffffu) {
            if (acc_nodes)
                atomicAdd(&a.cnt.search_nodes[acc_inst], acc_nodes);
            if (fm != INT_MAX)
                atomicMin(&a.cnt.fnext_off[acc_inst], fm);
            for (int m = 0; FUSE && m < acc_J; ++m)
                if (lowc[m]) {
                    atomicAdd(&a.fuse.low[(size_t)acc_inst * FUSE_K + m], (unsigned long long)lowc[m]);
                    lowc[m] = 0;
                }
        }
        acc_nodes = 0;
        fmin = INT_MAX;
    };

    for (;;) {
        int h = 0;
        if (lane == 0)
            h = atomicAdd(&a.ctrl->head, chunk);
        h = __shfl_sync(FULL, h, 0);
        if (h >= n_in)
            break;
        const int end = min(h + chunk, n_in);
        int i = h;
        while (i < end) {
            // the run of records [i, i+cnt) that belong to one instance
            const int idx = i + lane;
            const bool v = idx < end;
            Rec<W> r;
            if (v)
                r = load_rec<W>(a, frontier, n_act, n_front, act, in, idx);
            const unsigned inst = v ? r.inst : 0xffffffffu;
            const unsigned inst0 = __shfl_sync(FULL, inst, 0);
            const unsigned same = __ballot_sync(FULL, v && inst == inst0);
            const int cnt = (same == FULL) ? 32 : (__ffs(~same) - 1);
            // an instance whose node budget ran out, or that already found
            // its goal in first-solution mode, is dropped
            const unsigned long long left = a.cnt.budget_left[inst0];
            const bool budgeted = left != ~0ull;
            const bool watch = budgeted || first_only;
            const bool dropped = watch && *(volatile unsigned *)&a.cnt.aborted[inst0];
            if (lane < cnt && !dropped) {
                if constexpr (PDB) {
                    const u128 e = pdb_encode<W>(r.b, *pi);
                    uint32_t vb;
                    pdb_h(a.pdb, *pi, (uint64_t)(e >> 64), &vb);
                    stk.put(lane, e, sm_from_rec<W>(r.meta) | vb, r.origin);
                } else if constexpr (BF) {
                    const uint32_t sm = sm_from_rec<W>(r.meta);
                    stk.put(lane, to_blank_frame(r.b, sm & 127u), sm, r.origin);
                } else {
                    stk.put(lane, r.b, FM ? fm_from_rec(r.meta) : sm_from_rec<W>(r.meta), r.origin);
                }
            }
            if constexpr (FM || BF) {
                // the slots of these steps assume at most three children per
                // node: a record without a parent move (only the goal can be
                // one, the splitter expands every other root) fails the call
                const bool root = lane < cnt && !dropped && m_last(r.meta) == LAST_NONE && r.b != GOAL;
                if (__any_sync(FULL, root) && lane == 0)
                    atomicOr(&a.ctrl->err, ERR_INTERNAL);
            }
            int top = dropped ? 0 : cnt;
            if (inst0 != acc_inst) {
                publish();
                acc_inst = inst0;
                acc_J = (FUSE && a.fuse.jump) ? a.fuse.jump[inst0] : 0;
            }
            const int J = FUSE ? acc_J : 0;
            __syncwarp();
            // nodes popped in this run: a 32-bit count per round, folded into
            // the 64-bit total every 32 rounds (at most 1024 in between)
            unsigned long long nodes = 0, flushed = 0;
            unsigned n32 = 0;

            while (top > 0 || (OVF && ovf_n > 0)) {
                if (OVF && top == 0) {
                    // refill from the overflow stack (its most recent spill)
                    const int k = min(ovf_n, S / 2);
                    for (int j = lane; j < k; j += 32) {
                        SB bb;
                        uint32_t mm, oo;
                        ovf.get(ovf_n - k + j, bb, mm, oo);
                        stk.put(j, bb, mm, oo);
                    }
                    ovf_n -= k;
                    top = k;
                    __syncwarp();
                }
                const int n = min(32, top);
                if (top + 3 * n > S) {
                    // keep room for up to 4n children (an instance root has
                    // four): move the oldest entries to the overflow stack,
                    // or hand them to the next pass when it is full, and move
                    // the rest down. Afterwards top <= max(n, S/2), so
                    // top + 3n <= S for S >= 192 KN.
                    const int k = min(top - n, S / 2);
                    if (lane == 0)
                        atomicAdd(&a.ctrl->spills, 1ull);
                    if (OVF && ovf_n + k <= a.ovf_cap) {
                        for (int j = lane; j < k; j += 32) {
                            SB bb;
                            uint32_t mm, oo;
                            stk.get(j, bb, mm, oo);
                            ovf.put(ovf_n + j, bb, mm, oo);
                        }
                        ovf_n += k;
                    } else {
                        hand_back_stack<W, S, PDB>(a, out, stk, 0, k, inst0, lane, pi, FM, BF);
                    }
                    __syncwarp();
                    for (int j0 = 0; j0 < top - k; j0 += 32) {
                        const int j = j0 + lane;
                        const bool ok = j < top - k;
                        SB bb = 0;
                        uint32_t mm = 0, oo = 0;
                        if (ok)
                            stk.get(k + j, bb, mm, oo);
                        __syncwarp();
                        if (ok)
                            stk.put(j, bb, mm, oo);
                        __syncwarp();
                    }
                    top -= k;
                }
                // pop: lane l takes entry top - n + l
                const bool act = lane < n;
                SB b;
                uint32_t mt, org;
                // every lane reads an entry unconditionally (a lane past n reads an
                // entry below S: lane < 32 <= S when n = top, and top - 1
                // otherwise); the lanes past n push nothing and count nothing
                stk.get(top - n + lane, b, mt, org);
                top -= n;
                n32 += (unsigned)n;
                __syncwarp();

                // (in the blank's frame, a board whose blank is elsewhere can
                // read as the goal)
                const bool goal = act && (b == GOAL) && (!BF || (mt & 127u) == 0u);
                const unsigned gmask = __ballot_sync(FULL, goal);
                if (gmask) {
                    const unsigned o = warp_min_u32(goal ? org : 0xffffffffu);
                    if (lane == 0) {
                        atomicAdd(&a.cnt.goals[inst0], (unsigned long long)__popc(gmask));
                        atomicMin(&a.cnt.goal_origin[inst0], o);
                        // first-solution mode stops the instance, unless this
                        // step fuses several of its thresholds: a fused step
                        // runs to completion (the counts of its lower
                        // thresholds need the whole pass)
                        if (first_only && J == 0)
                            atomicOr(&a.cnt.aborted[inst0], ABORT_FOUND);
                    }
                    if (FUSE && J && goal) {
                        // a goal at slack s belongs to iteration J - s/2 of the step
                        const int j = J - (int)(FM ? (mt >> 9) & 63u : (mt >> 12) & 127u);
                        if (j >= 0) {
                            atomicAdd(&a.fuse.goals[(size_t)inst0 * FUSE_K + j], 1ull);
                            atomicMin(&a.fuse.origin[(size_t)inst0 * FUSE_K + j], org);
                        }
                    }
                }
                int base = top;
                const int s = FM ? (int)((mt >> 8) & 127u) : (int)((mt >> 11) & 255u);
                if constexpr (FUSE) {
                    // popped nodes above the lower limits of the step
                    const unsigned hm = (unsigned)s >> 1;
                    if (J && act && hm < (unsigned)J)
                        lowp += 1ull << (8 * hm);
                }
                if constexpr (FM) {
                    // the four moves at once (see FourMoves)
                    const uint32_t mq = mt;
                    const uint32_t p = mq & 15u;
                    const uint2 e01 = fmtab[p], e23 = fmtab[16 + p];
                    const uint4 e = make_uint4(e01.x, e01.y, e23.x, e23.y);
                    const uint64_t bq = (uint64_t)b;
                    const uint32_t G = __byte_perm((uint32_t)bq, (uint32_t)(bq >> 32), e.x);
                    // byte m's low nibble: the tile that move m slides into the blank
                    const uint32_t Y = (G & e.y) | ((G >> 4) & ~e.y);
                    const uint32_t X = (Y & 0x0F03030Fu) ^ 0x0F030000u;
                    const uint32_t away4 = (e.z - X) & FM_BIT7;
                    const uint32_t allowed4 = (act && !goal) ? (e.w & ~mq) : 0u;
                    const uint32_t low4 = (mq & 0x7E00u) ? 0u : FM_BIT7;  // slack < 2
                    const uint32_t push4 = allowed4 & ~(away4 & low4);
                    prn |= allowed4 & away4 & low4;
                    const uint32_t keep = mq & 0x7F0Fu;  // blank position and slack
                    // slots: this lane's children go to consecutive entries from
                    // base + the prefix of the per-lane counts (from their
                    // bit-sliced ballots); sa is the next one's shared-window address
                    // (every node here has a parent move, so c <= 3: two slices)
                    const unsigned c = __popc(push4);
                    const unsigned B0 = __ballot_sync(FULL, c & 1u), B1 = __ballot_sync(FULL, c & 2u);
                    uint32_t sa = 0;
                    if constexpr (FM)
                        sa = stk.addr(base + __popc(B0 & lt) + 2 * __popc(B1 & lt));
                    base += (int)__reduce_add_sync(FULL, c);
                    // the children: move m writes its tile t into the blank's field
                    // (zero) and clears the neighbour's (which holds t), i.e. adds t
                    // times a per-position constant to each 32-bit half (16^p less
                    // 16^np; a field never carries or borrows), one multiply-add; the
                    // tile and the away bit of byte m are read with byte dot
                    // products, so the step's arithmetic runs on the multiply-add
                    // pipe rather than on the integer ALU pipe, which the tests
                    // and the bit logic above already keep busy
                    const uint32_t Yc = Y & 0x0F0F0F0Fu;
                    const uint2 l01 = fmtab[32 + p], l23 = fmtab[48 + p], h01 = fmtab[64 + p], h23 = fmtab[80 + p];
                    const uint4 ml = make_uint4(l01.x, l01.y, l23.x, l23.y), mh = make_uint4(h01.x, h01.y, h23.x, h23.y);
                    const uint32_t mlo[4] = {ml.x, ml.y, ml.z, ml.w}, mhi[4] = {mh.x, mh.y, mh.z, mh.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t t = (uint32_t)__dp4a(Yc, ebyte[m], 0u);
                        const uint32_t clo = t * mlo[m] + (uint32_t)bq, chi = t * mhi[m] + (uint32_t)(bq >> 32);
                        const B child = ((uint64_t)chi << 32) | clo;
                        // the child's blank, its excluded move (the inverse of m)
                        // and its slack (s - 2 when the tile moved away, else s:
                        // the signed dot product of the away bits with e4[m])
                        const uint32_t cm = (uint32_t)__dp4a(
                            (int)away4, e4[m], (int)(keep + (uint32_t)move_off<W>(m) + (0x80u << (8 * (3 - m)))));
                        const uint32_t pb = push4 & (0x80u << (8 * m));
                        if constexpr (FM)
                            stk.put_if(pb, sa, child, cm, org);
                        sa += pb ? 16u : 0u;
                    }

                } else if constexpr (BF) {
                    // the 24-puzzle in the blank's frame (see BlankFrame): the
                    // position's table row gives the legal moves (bits 28..31
                    // of word 0) and, word m, whether move m's tile slides away
                    // from its goal cell (bit t)
                    const uint32_t sh_p = mt & 127u;
                    const LutRow<W> row = lut_row_sh<W>(lut, sh_p);
                    const uint32_t rw[4] = {row.v.x, row.v.y, row.v.z, row.v.w};
                    const uint32_t w0 = (uint32_t)b, w1 = (uint32_t)(b >> 32), w2 = (uint32_t)(b >> 64),
                                   w3 = (uint32_t)(b >> 96);
                    // the tiles of the neighbours up, left, right, down (fields 20, 24, 1, 5)
                    const uint32_t t[4] = {(w3 >> 4) & 31u, w3 >> 24, (w0 >> 5) & 31u, (w0 >> 25) & 31u};
                    // moves other than the inverse of the parent's (bits 7..10 of mt)
                    const uint32_t ok4 = (act && !goal) ? ((rw[0] >> 28) & ~(mt >> 7) & 15u) : 0u;
                    uint32_t aw[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        aw[m] = (rw[m] >> t[m]) & 1u;
                    const uint32_t away4 = aw[0] + 2u * aw[1] + 4u * aw[2] + 8u * aw[3];
                    const uint32_t cut4 = (s < 2) ? (ok4 & away4) : 0u;  // children past the limit
                    const uint32_t push4 = ok4 & ~cut4;
                    if (cut4)
                        fmin = min(fmin, 2 - s);
                    // slots: this lane's children go to sp, sp + 1, ... (the
                    // prefix of the per-lane counts, from their bit-sliced ballots)
                    const unsigned c = __popc(push4);
                    // (every node here has a parent move, so c <= 3: two slices)
                    const unsigned B0 = __ballot_sync(FULL, c & 1u), B1 = __ballot_sync(FULL, c & 2u);
                    int sp = base + __popc(B0 & lt) + 2 * __popc(B1 & lt);
                    base += (int)__reduce_add_sync(FULL, c);
                    // the children: the board turned left by 25 (up) or 5 bits
                    // (left), right by 5 (right) or 25 (down); field 0 then holds
                    // the tile (it becomes the blank: subtract it) and the
                    // parent's blank cell, now field 5, 1, 24 or 20, holds 0 (it
                    // gets the tile: add it). A left turn also brings the low 3
                    // bits of the tile's old field to bits 125..127 (subtract
                    // them); a right turn wraps field 0, which is zero. Every
                    // field update is thus one multiply-add.
                    const uint32_t w3s = w3 << 3;  // field 24 at the top of a word
                    uint32_t c0[4], c1[4], c2[4], c3[4];
                    c0[0] = __funnelshift_l(w3s, w0, 25) + t[0] * ((1u << 25) - 1u);
                    c1[0] = __funnelshift_l(w0, w1, 25);
                    c2[0] = __funnelshift_l(w1, w2, 25);
                    c3[0] = __funnelshift_l(w2, w3, 25) - t[0] * (1u << 29);
                    c0[1] = __funnelshift_l(w3s, w0, 5) + t[1] * 31u;
                    c1[1] = __funnelshift_l(w0, w1, 5);
                    c2[1] = __funnelshift_l(w1, w2, 5);
                    c3[1] = __funnelshift_l(w2, w3, 5) - t[1] * (1u << 29);
                    c0[2] = __funnelshift_r(w0, w1, 5) - t[2];
                    c1[2] = __funnelshift_r(w1, w2, 5);
                    c2[2] = __funnelshift_r(w2, w3, 5);
                    c3[2] = (w3 >> 5) + t[2] * (1u << 24);
                    c0[3] = __funnelshift_r(w0, w1, 25) - t[3];
                    c1[3] = __funnelshift_r(w1, w2, 25);
                    c2[3] = __funnelshift_r(w2, w3, 25);
                    c3[3] = (w3 >> 25) + ((w0 & 0x01FFFFFFu) | t[3]) * 16u;
                    // the child's blank, its excluded move (the inverse of m) and
                    // its slack (s - 2 when the tile moved away, else s)
                    const uint32_t keep = mt & ~(15u << 7);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t pb = (push4 >> m) & 1u;
                        const uint32_t cm = aw[m] * (0u - (2u << 11)) +
                                            (keep + (uint32_t)(BITS * move_off<W>(m)) + ((1u << (3 - m)) << 7));
                        const B child = ((u128)c3[m] << 96) | ((u128)c2[m] << 64) | ((u128)c1[m] << 32) | c0[m];
                        if constexpr (BF)
                            stk.put_if(pb, sp, child, cm, org);
                        sp += (int)pb;
                    }
                } else {
                const uint32_t sh_p = mt & 127u;
                const unsigned allowed =
                    (act && !goal) ? (LegalMoves<W>::at_sh(sh_p) & ~((mt >> 7) & 15u)) : 0u;
                const bool low = s < 2;
                const uint32_t sbase = mt & (255u << 11);
                bool pruned = false;
                if constexpr (PDB) {
                    // b holds the inverse board (high half) and the slot board
                    // (low half); the step's direction comes from the moved
                    // tile's group table, h_g mod 4 from the metadata
                    const uint64_t sb = (uint64_t)b, inv = (uint64_t)(b >> 64);
                    const uint32_t vkeep = mt & PDB_VMASK;
                    bool bad = false;
                    // first the four table reads, issued together so that their
                    // latencies overlap (the search waits on them, not on issue),
                    // then the children
                    uint32_t jm[4], vm[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t sh_np = sh_p + (uint32_t)(4 * move_off<W>(m));
                        // slot of the tile that slides into the blank (an off-board
                        // offset reads slot 0, whose entry is zero)
                        jm[m] = BoardOps<W>::tile(sb, sh_np);
                        vm[m] = 0;
                        if ((allowed >> m) & 1u) {
                            const PdbSlot sl = pi->slot[jm[m]];
                            // the tile moves np -> p, the blank p -> np
                            const uint64_t dd = (uint64_t)((sh_p ^ sh_np) >> 2);
                            const uint64_t cinv = inv ^ (dd << (4 * jm[m])) ^ dd;
                            uint64_t f;
                            asm("shr.b64 %0, %1, %2;" : "=l"(f) : "l"(cinv), "r"(sl.goff));
                            // field | np << width, as one multiply-add (the field is below mask + 1)
                            const uint32_t idx = ((uint32_t)f & sl.mask) + (sh_np >> 2) * (sl.mask + 1u);
                            vm[m] = __ldg(a.pdb.tab + sl.base + idx);
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const bool legal = (allowed >> m) & 1u;
                        const uint32_t sh_np = sh_p + (uint32_t)(4 * move_off<W>(m));
                        const uint32_t j = jm[m];
                        const PdbSlot sl = pi->slot[j];
                        const uint64_t dd = (uint64_t)((sh_p ^ sh_np) >> 2);
                        const uint64_t cinv = inv ^ (dd << (4 * j)) ^ dd;
                        const uint32_t sh_q = (m < 2) ? sh_np : sh_p;  // lower of the two fields
                        const uint64_t csb = BoardOps<W>::flip(sb, j * move_mul<W>(m), sh_q);
                        const uint32_t v = vm[m];
                        const uint32_t vold = mt >> sl.vsh;
                        // h_g rose by 1 (dv = 1) or fell by 1 (dv = 3); any other
                        // dv is an inconsistent table: it counts as a rise (so a
                        // subtree stays finite) and fails the call
                        const uint32_t dv = (v - vold) & 3u;
                        const bool away = dv != 3u;
                        bad |= legal && dv != 1u && dv != 3u;
                        const bool push = legal && !(away && low);
                        pruned |= legal && away && low;
                        const uint32_t cm = ((sh_np + sbase + ((1u << (3 - m)) << 7)) - (away ? (2u << 11) : 0u)) |
                                            (vkeep ^ (((v ^ vold) & 3u) << sl.vsh));
                        const unsigned pm = __ballot_sync(FULL, push);
                        if (push)
                            stk.put(base + __popc(pm & lt), ((u128)cinv << 64) | csb, cm, org);
                        base += __popc(pm);
                    }
                    if (__any_sync(FULL, bad) && lane == 0)
                        atomicOr(&a.ctrl->err, ERR_INTERNAL);
                } else {
                const LutRow<W> row = lut_row_sh<W>(lut, sh_p);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const bool legal = (allowed >> m) & 1u;
                    // field offset of the tile that slides into the blank
                    const uint32_t sh_np = sh_p + (uint32_t)(BITS * move_off<W>(m));
                    const unsigned t = BoardOps<W>::tile(b, sh_np);
                    // h changes by +1 (away from the tile's goal cell) or -1
                    // and g by +1, so the child's slack is s - 2 or s
                    const bool away = away_bit<W>(row, m, t);
                    const bool push = legal && !(away && low);
                    pruned |= legal && away && low;
                    const uint32_t sh_q = (m < 2) ? sh_np : sh_p;  // lower of the two fields
                    const B child = BoardOps<W>::flip(b, t * move_mul<W>(m), sh_q);
                    const uint32_t cm = (sh_np + sbase + ((1u << (3 - m)) << 7)) - (away ? (2u << 11) : 0u);
                    const unsigned pm = __ballot_sync(FULL, push);
                    if (push)
                        stk.put(base + __popc(pm & lt), child, cm, org);
                    base += __popc(pm);
                }
                }
                if (pruned)
                    fmin = min(fmin, 2 - s);
                }
                top = base;
                __syncwarp();

                if (((++rounds) & 31) == 0) {
                    nodes += n32;
                    n32 = 0;
                    if (FUSE && J)
                        flush_low(J);
                    if (first_only && J == 0) {
                        int found = 0;
                        if (lane == 0)
                            found = (*(volatile unsigned *)&a.cnt.aborted[inst0] & ABORT_FOUND) != 0;
                        if (__shfl_sync(FULL, found, 0)) {
                            top = 0;
                            ovf_n = 0;
                            break;
                        }
                    }
                    if (budgeted) {
                        // publish this run's count; past the budget the
                        // instance's remaining work is dropped
                        int over = 0;
                        if (lane == 0) {
                            const unsigned long long before = atomicAdd(&a.cnt.search_nodes[inst0], nodes - flushed);
                            over = before + (nodes - flushed) > left;
                            if (over)
                                atomicOr(&a.cnt.aborted[inst0], ABORT_BUDGET);
                        }
                        flushed = nodes;
                        if (__shfl_sync(FULL, over, 0)) {
                            top = 0;
                            ovf_n = 0;
                            break;
                        }
                    }
                    if (rounds >= a.tune.min_rounds) {
                        // hand back once enough warps have run dry and the
                        // pass has run long enough to pay for another one
                        int go = 0;
                        if (lane == 0 && *(volatile int *)&a.ctrl->exited >= a.tune.exit_threshold)
                            go = global_ns() - *(volatile unsigned long long *)&a.ctrl->t_start >=
                                 (unsigned long long)a.tune.min_pass_ns;
                        // serving: the step's time slice is over
                        if (lane == 0 && !go && slice_over(a))
                            go = 1;
                        if (__shfl_sync(FULL, go, 0)) {
                            stop = true;
                            break;
                        }
                    }
                }
            }
            // this run's counts
            nodes += n32;
            if (FUSE && J)
                flush_low(J);
            acc_nodes += nodes - flushed;
            tot_nodes += nodes;
            if (budgeted)
                publish();
            if (stop) {
                hand_back_stack<W, S, PDB>(a, out, stk, 0, top, inst0, lane, pi, FM, BF);
                if (OVF)
                    hand_back_stack<W, S, PDB>(a, out, ovf, 0, ovf_n, inst0, lane, pi, FM, BF);
                ovf_n = 0;
                hand_back_records<W>(a, frontier, n_act, n_front, act, in, out, i + cnt, end, lane);
                // input that no warp has taken yet goes back too (a stop at
                // the end of a serving time slice can come before the input
                // is exhausted; otherwise nothing is left here)
                for (;;) {
                    int h2 = 0;
                    if (lane == 0)
                        h2 = atomicAdd(&a.ctrl->head, chunk);
                    h2 = __shfl_sync(FULL, h2, 0);
                    if (h2 >= n_in)
                        break;
                    hand_back_records<W>(a, frontier, n_act, n_front, act, in, out, h2, min(h2 + chunk, n_in), lane);
                }
                break;
            }
            i += cnt;
        }
        if (stop)
            break;
    }
    publish();
    if (!stop && lane == 0)
        atomicAdd(&a.ctrl->exited, 1);
    // the last warp of a block publishes the block's end time and node
    // count; the last block to finish closes the pass
    if (lane == 0) {
        atomicMax(&s_t_end, global_ns());
        atomicAdd(&s_nodes, tot_nodes);
        __threadfence();
        if (atomicAdd(&s_warps_done, 1) == (int)(blockDim.x >> 5) - 1) {
            __threadfence();
            atomicMax(&a.ctrl->t_end, *(volatile unsigned long long *)&s_t_end);
            atomicAdd(&a.ctrl->search_nodes_total, *(volatile unsigned long long *)&s_nodes);
            __threadfence();
            if (atomicAdd(&a.ctrl->done_warps, 1) == (int)gridDim.x - 1) {
                __threadfence();
                end_of_pass<W>(a);
            }
        }
    }
}

// ---------------------------------------------------------------------
// Block-per-subtree search (bpida_config.variant = 6), the other mode of the
// autotuner: all warps of a block share one stack of S entries per warp, as
// in Algorithm 1 with a block larger than a warp. Each round pops up to
// blockDim nodes (one per thread); a thread's children go to slots from a
// block-wide prefix of the per-thread counts (bit-sliced ballots within a
// warp, warp totals through shared memory), with block barriers between the
// pop and the pushes. Everything else is as in k_search: runs of records of
// one instance from the pass's queue, node budget and first-solution checks
// every 32 rounds, hand-back once enough warps have run dry. 8- and
// 15-puzzle, Manhattan distance.
// ---------------------------------------------------------------------
template <int W, int S>
__global__ void k_search_block(const Dev<W> a)
{
    typedef typename Geo<W>::B B;
    static_assert(W <= 4, "block mode: 8- and 15-puzzle");
    constexpr int BITS = Geo<W>::BITS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cnt[32];
    __shared__ int s_h, s_first, s_flag, s_fmin;
    __shared__ unsigned s_inst;
    unsigned char *lut = smem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nw = nthr >> 5;
    const int SB = S * nw;  // the block's stack entries
    if (tid == 0)
        atomicMin(&a.ctrl->t_start, global_ns());
    SharedLut<W>::load(lut, a.lut);
    if (tid == 0)
        s_fmin = INT_MAX;
    __syncthreads();
    WarpStack<W> stk;
    stk.init(smem + SearchSmem<W>::TABLES, SB);
    const Rec<W> *in = a.ctrl->qi ? a.q1 : a.q0;
    Rec<W> *out = a.ctrl->qi ? a.q0 : a.q1;
    const bool frontier = a.ctrl->first_pass != 0;
    const int n_act = a.ctrl->n_active;
    const int n_front = a.ctrl->n_front;
    const unsigned *act_list = a.ctrl->cur ? a.act1 : a.act0;
    const bool first_only = a.desc->first_only != 0;
    const unsigned lt = (1u << lane) - 1u;
    const B GOAL = goal_board<W>();
    const int n_in = a.ctrl->n_in;
    const int chunk = max(1, min(nthr, n_in / (int)(gridDim.x * 4)));
    int rounds = 0;
    bool stop = false;
    unsigned acc_inst = 0xffffffffu;
    unsigned long long acc_nodes = 0, tot_nodes = 0;  // the same in every thread
    int fmin = INT_MAX;
    // block-wide: publishes the counters of acc_inst (every thread calls it)
    auto publish = [&]() {
        const int fm = warp_min_int(fmin);
        if (lane == 0 && fm != INT_MAX)
            atomicMin(&s_fmin, fm);
        __syncthreads();
        if (tid == 0 && acc_inst != 0xffffffffu) {
            if (acc_nodes)
                atomicAdd(&a.cnt.search_nodes[acc_inst], acc_nodes);
            if (s_fmin != INT_MAX)
                atomicMin(&a.cnt.fnext_off[acc_inst], s_fmin);
        }
        __syncthreads();
        if (tid == 0)
            s_fmin = INT_MAX;
        acc_nodes = 0;
        fmin = INT_MAX;
    };
    // block-wide: stack entries [from, from + k) to the next pass
    auto hand_back = [&](int from, int k, unsigned inst) {
        if (k <= 0)
            return;
        if (tid == 0)
            s_h = atomicAdd(&a.ctrl->out_count, k);
        __syncthreads();
        const int base = s_h;
        __syncthreads();
        if (base + k > a.Q) {
            if (tid == 0)
                atomicOr(&a.ctrl->err, ERR_QUEUE);
            return;
        }
        for (int j = tid; j < k; j += nthr) {
            B b;
            uint32_t m, o;
            stk.get(from + j, b, m, o);
            Rec<W> r;
            r.b = b;
            r.meta = rec_from_sm<W>(m);
            r.inst = inst;
            r.origin = o;
            r.pm = 0;
            out[base + j] = r;
        }
    };
    auto hand_back_input = [&](int from, int to) {
        const int k = to - from;
        if (k <= 0)
            return;
        if (tid == 0)
            s_h = atomicAdd(&a.ctrl->out_count, k);
        __syncthreads();
        const int base = s_h;
        __syncthreads();
        if (base + k > a.Q) {
            if (tid == 0)
                atomicOr(&a.ctrl->err, ERR_QUEUE);
            return;
        }
        for (int j = tid; j < k; j += nthr)
            out[base + j] = load_rec<W>(a, frontier, n_act, n_front, act_list, in, from + j);
    };

    for (;;) {
        if (tid == 0)
            s_h = atomicAdd(&a.ctrl->head, chunk);
        __syncthreads();
        const int h = s_h;
        __syncthreads();
        if (h >= n_in)
            break;
        const int end = min(h + chunk, n_in);
        int i = h;
        while (i < end) {
            // the run of records [i, i + cnt) that belong to one instance
            const int idx = i + tid;
            const bool v = idx < end;
            Rec<W> r;
            if (v)
                r = load_rec<W>(a, frontier, n_act, n_front, act_list, in, idx);
            if (tid == 0) {
                s_inst = r.inst;
                s_first = nthr;
            }
            __syncthreads();
            const unsigned inst0 = s_inst;
            if (!(v && r.inst == inst0))
                atomicMin(&s_first, tid);
            __syncthreads();
            const int cnt = s_first;
            const unsigned long long left = a.cnt.budget_left[inst0];
            const bool budgeted = left != ~0ull;
            if (tid == 0)
                s_flag = (budgeted || first_only) && *(volatile unsigned *)&a.cnt.aborted[inst0];
            __syncthreads();
            const bool dropped = s_flag != 0;
            if (tid < cnt && !dropped)
                stk.put(tid, r.b, sm_from_rec<W>(r.meta), r.origin);
            int top = dropped ? 0 : cnt;
            if (inst0 != acc_inst) {
                publish();
                acc_inst = inst0;
            }
            __syncthreads();
            unsigned long long nodes = 0, flushed = 0;
            while (top > 0) {
                const int n = min(nthr, top);
                if (top + 3 * n > SB) {
                    // room for 4n children: the oldest entries go to the next
                    // pass, the rest move down (afterwards top <= max(n, SB/2),
                    // so top + 3n <= SB for SB >= 6 blockDim)
                    const int k = min(top - n, SB / 2);
                    if (tid == 0)
                        atomicAdd(&a.ctrl->spills, 1ull);
                    hand_back(0, k, inst0);
                    __syncthreads();
                    for (int j0 = 0; j0 < top - k; j0 += nthr) {
                        const int j = j0 + tid;
                        const bool ok = j < top - k;
                        B bb = 0;
                        uint32_t mm = 0, oo = 0;
                        if (ok)
                            stk.get(k + j, bb, mm, oo);
                        __syncthreads();
                        if (ok)
                            stk.put(j, bb, mm, oo);
                        __syncthreads();
                    }
                    top -= k;
                }
                const bool act = tid < n;
                B b = 0;
                uint32_t mt = 0, org = 0;
                if (act)
                    stk.get(top - n + tid, b, mt, org);
                top -= n;
                nodes += (unsigned long long)n;
                __syncthreads();
                const bool goal = act && (b == GOAL);
                const unsigned gmask = __ballot_sync(FULL, goal);
                if (gmask) {
                    const unsigned o = warp_min_u32(goal ? org : 0xffffffffu);
                    if (lane == 0) {
                        atomicAdd(&a.cnt.goals[inst0], (unsigned long long)__popc(gmask));
                        atomicMin(&a.cnt.goal_origin[inst0], o);
                        if (first_only)
                            atomicOr(&a.cnt.aborted[inst0], ABORT_FOUND);
                    }
                }
                const uint32_t sh_p = mt & 127u;
                const int s = (int)((mt >> 11) & 255u);
                const unsigned allowed = (act && !goal) ? (LegalMoves<W>::at_sh(sh_p) & ~((mt >> 7) & 15u)) : 0u;
                const bool low = s < 2;
                const LutRow<W> row = lut_row_sh<W>(lut, sh_p);
                unsigned push4 = 0;
                bool pruned = false;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const bool legal = (allowed >> m) & 1u;
                    const unsigned t = BoardOps<W>::tile(b, sh_p + (uint32_t)(BITS * move_off<W>(m)));
                    const bool away = away_bit<W>(row, m, t);
                    push4 |= (legal && !(away && low)) ? (1u << m) : 0u;
                    pruned |= legal && away && low;
                }
                if (pruned)
                    fmin = min(fmin, 2 - s);
                // slots: the block-wide prefix of the per-thread child counts
                const unsigned c = __popc(push4);
                const unsigned B0 = __ballot_sync(FULL, c & 1u), B1 = __ballot_sync(FULL, c & 2u),
                               B2 = __ballot_sync(FULL, c & 4u);
                const int off = __popc(B0 & lt) + 2 * __popc(B1 & lt) + 4 * __popc(B2 & lt);
                if (lane == 0)
                    s_cnt[warp] = __popc(B0) + 2 * __popc(B1) + 4 * __popc(B2);
                __syncthreads();
                int before = 0, total = 0;
                for (int w = 0; w < nw; ++w) {
                    const int x = s_cnt[w];
                    before += w < warp ? x : 0;
                    total += x;
                }
                int sp = top + before + off;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if ((push4 >> m) & 1u) {
                        const uint32_t sh_np = sh_p + (uint32_t)(BITS * move_off<W>(m));
                        const unsigned t = BoardOps<W>::tile(b, sh_np);
                        const bool away = away_bit<W>(row, m, t);
                        const B child = BoardOps<W>::flip(b, t * move_mul<W>(m), (m < 2) ? sh_np : sh_p);
                        const uint32_t cm =
                            (sh_np + (mt & (255u << 11)) + ((1u << (3 - m)) << 7)) - (away ? (2u << 11) : 0u);
                        stk.put(sp, child, cm, org);
                        ++sp;
                    }
                }
                top += total;
                __syncthreads();

                if (((++rounds) & 31) == 0) {
                    // 1: first solution found, 2: over the node budget, 3: hand back
                    if (tid == 0) {
                        int f = 0;
                        if (first_only && (*(volatile unsigned *)&a.cnt.aborted[inst0] & ABORT_FOUND))
                            f = 1;
                        if (!f && budgeted) {
                            const unsigned long long before_n = atomicAdd(&a.cnt.search_nodes[inst0], nodes - flushed);
                            if (before_n + (nodes - flushed) > left) {
                                atomicOr(&a.cnt.aborted[inst0], ABORT_BUDGET);
                                f = 2;
                            }
                        }
                        if (!f && rounds >= a.tune.min_rounds &&
                            *(volatile int *)&a.ctrl->exited >= a.tune.exit_threshold &&
                            global_ns() - *(volatile unsigned long long *)&a.ctrl->t_start >=
                                (unsigned long long)a.tune.min_pass_ns)
                            f = 3;
                        if (!f && rounds >= a.tune.min_rounds && slice_over(a))
                            f = 3;
                        s_flag = f;
                    }
                    if (budgeted)
                        flushed = nodes;
                    __syncthreads();
                    const int f = s_flag;
                    __syncthreads();
                    if (f == 1 || f == 2) {
                        top = 0;
                        break;
                    }
                    if (f == 3) {
                        stop = true;
                        break;
                    }
                }
            }
            acc_nodes += nodes - flushed;
            tot_nodes += nodes;
            if (budgeted)
                publish();
            if (stop) {
                hand_back(0, top, inst0);
                hand_back_input(i + cnt, end);
                // input no block has taken yet goes back too
                for (;;) {
                    if (tid == 0)
                        s_h = atomicAdd(&a.ctrl->head, chunk);
                    __syncthreads();
                    const int h2 = s_h;
                    __syncthreads();
                    if (h2 >= n_in)
                        break;
                    hand_back_input(h2, min(h2 + chunk, n_in));
                }
                break;
            }
            i += cnt;
        }
        if (stop)
            break;
    }
    publish();
    if (tid == 0) {
        if (!stop)
            atomicAdd(&a.ctrl->exited, nw);
        atomicMax(&a.ctrl->t_end, global_ns());
        atomicAdd(&a.ctrl->search_nodes_total, tot_nodes);
        __threadfence();
        if (atomicAdd(&a.ctrl->done_warps, 1) == (int)gridDim.x - 1) {
            __threadfence();
            end_of_pass<W>(a);
        }
    }
}

// ---------------------------------------------------------------------
// The paper's BPIDA* kernel, kept as an ablation of the design above
// (Algorithm 1 as printed): a block is one warp; each repetition pops
// #threads / #actions = 8 nodes and lane i applies action (i mod 4) to node
// i / 4; a child with f <= limit is pushed at a ballot-reserved slot
// (atomicPut), the others only lower f_next. Roots are assigned to blocks
// statically (block b takes an equal contiguous share of the root set) and
// there is no dynamic load balancing; the root set is sized from the
// previous iteration's work as for the main kernel. A full stack hands its
// oldest entries to another pass (rare), which keeps the kernel exact.
// ---------------------------------------------------------------------
template <int W, int S>
__global__ void __launch_bounds__(32) k_search_paper(const Dev<W> a)
{
    typedef typename Geo<W>::B B;
    constexpr int BITS = Geo<W>::BITS;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *lut = smem;
    if (threadIdx.x == 0)
        atomicMin(&a.ctrl->t_start, global_ns());
    SharedLut<W>::load(lut, a.lut);
    __syncthreads();
    const Rec<W> *in = a.ctrl->qi ? a.q1 : a.q0;
    Rec<W> *out = a.ctrl->qi ? a.q0 : a.q1;
    const bool frontier = a.ctrl->first_pass != 0;
    const int n_act = a.ctrl->n_active;
    const bool first_only = a.desc->first_only != 0;
    const int lane = threadIdx.x & 31;
    WarpStack<W> stk;
    stk.init(smem + SharedLut<W>::BYTES, S);
    const unsigned lt = (1u << lane) - 1u;
    const int j = lane >> 2, m = lane & 3;  // node j of the pop, action m
    const int n_in = a.ctrl->n_in;
    // static share of the roots
    const int share = (n_in + gridDim.x - 1) / gridDim.x;
    const int r0 = min(n_in, blockIdx.x * share), r1 = min(n_in, r0 + share);
    for (int i = r0; i < r1; ++i) {
        const Rec<W> r = load_rec<W>(a, frontier, n_act, a.ctrl->n_front, a.ctrl->cur ? a.act1 : a.act0, in, i);
        const unsigned inst0 = r.inst;
        const unsigned long long left = a.cnt.budget_left[inst0];
        const bool budgeted = left != ~0ull;
        if ((budgeted || first_only) && *(volatile unsigned *)&a.cnt.aborted[inst0])
            continue;
        if (lane == 0)
            stk.put(0, r.b, sm_from_rec<W>(r.meta), r.origin);
        int top = 1;
        __syncwarp();
        unsigned long long nodes = 0, flushed = 0;
        int fmin = INT_MAX;
        int rounds = 0;
        while (top > 0) {
            const int n = min(8, top);
            if (top + 3 * n > S) {
                const int k = min(top - n, S / 2);
                if (lane == 0)
                    atomicAdd(&a.ctrl->spills, 1ull);
                hand_back_stack<W, S>(a, out, stk, 0, k, inst0, lane);
                __syncwarp();
                for (int j0 = 0; j0 < top - k; j0 += 32) {
                    const int q = j0 + lane;
                    const bool ok = q < top - k;
                    B bb = 0;
                    uint32_t mm = 0, oo = 0;
                    if (ok)
                        stk.get(k + q, bb, mm, oo);
                    __syncwarp();
                    if (ok)
                        stk.put(q, bb, mm, oo);
                    __syncwarp();
                }
                top -= k;
            }
            // parallelPop: the top n nodes, four lanes per node
            const bool act = j < n;
            B b = 0;
            uint32_t mt = 0, org = 0;
            if (act)
                stk.get(top - n + j, b, mt, org);
            top -= n;
            nodes += (unsigned long long)n;
            __syncwarp();
            const bool goal = act && (b == goal_board<W>());
            const unsigned gmask = __ballot_sync(FULL, goal && m == 0);
            if (gmask) {
                const unsigned o = warp_min_u32((goal && m == 0) ? org : 0xffffffffu);
                if (lane == 0) {
                    atomicAdd(&a.cnt.goals[inst0], (unsigned long long)__popc(gmask));
                    atomicMin(&a.cnt.goal_origin[inst0], o);
                    if (first_only)
                        atomicOr(&a.cnt.aborted[inst0], ABORT_FOUND);
                }
            }
            const uint32_t sh_p = mt & 127u;
            const int s = (int)((mt >> 11) & 255u);
            const bool legal = act && !goal && ((LegalMoves<W>::at_sh(sh_p) & ~((mt >> 7) & 15u)) >> m & 1u);
            // the (threadID mod #actions)th action
            const uint32_t sh_np = sh_p + (uint32_t)(BITS * move_off<W>(m));
            const unsigned t = BoardOps<W>::tile(b, sh_np);
            const LutRow<W> row = lut_row_sh<W>(lut, sh_p);
            const bool away = away_bit<W>(row, m, t);
            const bool push = legal && !(away && s < 2);
            if (legal && away && s < 2)
                fmin = min(fmin, 2 - s);
            const B child = BoardOps<W>::flip(b, t * move_mul<W>(m), (m < 2) ? sh_np : sh_p);
            const uint32_t cm = (sh_np + (mt & (255u << 11)) + ((1u << (3 - m)) << 7)) - (away ? (2u << 11) : 0u);
            const unsigned pm = __ballot_sync(FULL, push);
            if (push)
                stk.put(top + __popc(pm & lt), child, cm, org);
            top += __popc(pm);
            __syncwarp();
            if (((++rounds) & 31) == 0 && (budgeted || first_only)) {
                int drop = 0;
                if (lane == 0) {
                    if (budgeted) {
                        const unsigned long long before = atomicAdd(&a.cnt.search_nodes[inst0], nodes - flushed);
                        if (before + (nodes - flushed) > left)
                            atomicOr(&a.cnt.aborted[inst0], ABORT_BUDGET);
                    }
                    drop = *(volatile unsigned *)&a.cnt.aborted[inst0] != 0;
                }
                if (budgeted)
                    flushed = nodes;
                if (__shfl_sync(FULL, drop, 0)) {
                    top = 0;
                    break;
                }
            }
        }
        fmin = warp_min_int(fmin);
        if (lane == 0) {
            atomicAdd(&a.cnt.search_nodes[inst0], nodes - flushed);
            atomicAdd(&a.ctrl->search_nodes_total, nodes);
            if (fmin != INT_MAX)
                atomicMin(&a.cnt.fnext_off[inst0], fmin);
        }
    }
    // the last warp closes the pass (hand-back only from full stacks)
    int last = 0;
    if (lane == 0) {
        atomicMax(&a.ctrl->t_end, global_ns());
        __threadfence();
        last = atomicAdd(&a.ctrl->done_warps, 1) == (int)gridDim.x - 1;
    }
    if (__shfl_sync(FULL, last, 0) && lane == 0) {
        __threadfence();
        end_of_pass<W>(a);
    }
}

// ---------------------------------------------------------------------
// Splitter: one block per problem; breadth-first, order-preserving
// expansion of the problem's root until the level holds `target` records
// (Algorithm 1's CreateRootSet, rebuilt every iteration). Nodes expanded
// here are counted here; the final level becomes the problem's frontier.
// Small levels stay in shared memory. The last block to finish computes the
// frontier offsets (exclusive scan of the record counts) and opens the
// step's first search pass, which reads the frontiers in place.
// ---------------------------------------------------------------------
template <int W> struct SplitShared {
    static constexpr int CAP = (W <= 4) ? 512 : 384;  // records per shared level buffer
};
static constexpr int SPLIT_THREADS = 512;

template <int W>
__device__ __forceinline__ bool last_block_done(unsigned *counter, int *s_last)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        *s_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*s_last) {
        __threadfence();
        return true;
    }
    return false;
}

template <int W, bool PDB = false>
__global__ void __launch_bounds__(SPLIT_THREADS) k_split(const Dev<W> a)
{
    typedef typename Geo<W>::B B;
    constexpr int BITS = Geo<W>::BITS;
    constexpr int SCAP = SplitShared<W>::CAP;
    __shared__ __align__(16) unsigned char lut[SharedLut<W>::BYTES];
    __shared__ Rec<W> lvl[2][SCAP];
    __shared__ int warp_sums[32];
    __shared__ int s_fmin, s_last, s_carry;
    __shared__ unsigned long long s_internal;
    __shared__ unsigned s_low[FUSE_MAX];  // expanded nodes with slack 2m, m < J (fused steps)

    Ctrl *ctrl = a.ctrl;
    const int k = blockIdx.x;
    const int n_active = ctrl->n_active;
    // serving: an instance whose open nodes were carried over continues its
    // iteration in this step (no split; its counters keep running)
    const unsigned inst_k = k < n_active ? (ctrl->cur ? a.act1 : a.act0)[k] : 0u;
    const bool continuing = k < n_active && a.slice && a.carry[inst_k];
    if (continuing) {
        __syncthreads();
        if (threadIdx.x == 0) {
            a.count[k] = 0;
            a.carry[inst_k] = 0;
        }
    } else if (k < n_active) {
        SharedLut<W>::load(lut, a.lut);
        const PdbInfo *pi = nullptr;
        if constexpr (PDB) {
            __shared__ PdbInfo s_pi;
            pdb_load_info(&s_pi, a.pdb.info);
            pi = &s_pi;
        }
        const unsigned inst = inst_k;
        const InstState<W> st = a.state[inst];
        Rec<W> *A = a.scratch + region_of(a, k, inst);
        Rec<W> *Bg = A + a.C;
        const B GOAL = goal_board<W>();
        if (threadIdx.x == 0) {
            Rec<W> r;
            r.b = st.root;
            r.meta = st.root_meta & M_NODE_MASK;
            if (r.b == GOAL)
                r.meta |= M_LEAF;
            r.inst = inst;
            r.origin = 0;
            r.pm = 0;
            lvl[0][0] = r;
            s_fmin = INT_MAX;
            s_internal = 0;
            a.cnt.search_nodes[inst] = 0;
            a.cnt.goals[inst] = 0;
            a.cnt.goal_origin[inst] = 0xffffffffu;
            a.cnt.aborted[inst] = 0;
            for (int m = 0; m < FUSE_MAX; ++m)
                s_low[m] = 0;
            if (a.fuse.jump)
                for (int j = 0; j < FUSE_K; ++j) {
                    a.fuse.goals[(size_t)inst * FUSE_K + j] = 0;
                    a.fuse.origin[(size_t)inst * FUSE_K + j] = 0xffffffffu;
                }
        }
        __syncthreads();
        const int J = a.fuse.jump ? st.jump : 0;

        const int T = max(1, (int)st.target);
        int cnt = 1, depth = 0;
        int expandable = (st.root == GOAL) ? 0 : 1;
        Rec<W> *cur = lvl[0];
        for (;;) {
            // the root is always expanded here (unless it is the goal): every
            // record the search kernel receives then has a parent move, so a
            // node there has at most three children
            if (expandable == 0 || depth >= 16 || 4 * cnt > a.C || (depth > 0 && cnt >= T))
                break;
            // the next level has at most 4*cnt records: shared memory if they fit
            Rec<W> *nxt;
            if (4 * cnt <= SCAP)
                nxt = (cur == lvl[0]) ? lvl[1] : lvl[0];
            else
                nxt = (cur == A) ? Bg : A;
            int outbase = 0, nonleaf = 0;
            int fmin = INT_MAX;
            unsigned long long internal = 0;
            for (int base = 0; base < cnt; base += blockDim.x) {
                const int j = base + threadIdx.x;
                Rec<W> r;
                r.meta = M_LEAF;
                const bool v = j < cnt;
                if (v)
                    r = cur[j];
                const bool leaf = v && (r.meta & M_LEAF);
                const bool exp = v && !leaf;
                Rec<W> c[4];
                int nc = 0, nl = 0;
                if (leaf) {
                    c[0] = r;
                    nc = 1;
                } else if (exp) {
                    internal += 1;
                    const int p = (int)m_blank(r.meta);
                    const int last = (int)m_last(r.meta);
                    const int s = m_slack(r.meta);
                    if (s < 2 * J)
                        atomicAdd(&s_low[s >> 1], 1u);
                    const uint32_t d = m_hi(r.meta);
                    const LutRow<W> e = SharedLut<W>::row(lut, p);
                    unsigned away4 = 0;
                    if constexpr (PDB) {
                        // the four moves' table reads together (see pdb_away4)
                        const uint64_t inv = pdb_inverse<W>(r.b, *pi);
                        uint32_t npm[4];
                        unsigned tm[4], legal = 0;
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const bool ok = e.legal(m) && last != 3 - m;
                            npm[m] = (uint32_t)(ok ? p + move_off<W>(m) : p);
                            tm[m] = ok ? tile_at<W>(r.b, (int)npm[m]) : 0u;
                            legal |= (ok ? 1u : 0u) << m;
                        }
                        away4 = pdb_away4(a.pdb, *pi, inv, (uint32_t)p, npm, tm, legal);
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (!e.legal(m) || last == 3 - m)
                            continue;
                        const int np = p + move_off<W>(m);
                        const unsigned t = tile_at<W>(r.b, np);
                        bool away;
                        if constexpr (PDB)
                            away = (away4 >> m) & 1u;
                        else
                            away = e.away(m, t);
                        const int s2 = away ? s - 2 : s;
                        if (s2 < 0) {
                            fmin = min(fmin, -s2);
                            continue;
                        }
                        const B x = (B)t;
                        Rec<W> ch;
                        ch.b = r.b + (x << (BITS * p)) - (x << (BITS * np));
                        ch.meta = (uint32_t)np | ((uint32_t)m << 5) | ((uint32_t)s2 << 8) | ((d + 1u) << 16);
                        if (ch.b == GOAL)
                            ch.meta |= M_LEAF;
                        else
                            ++nl;
                        ch.inst = inst;
                        ch.origin = 0;
                        ch.pm = r.pm | ((uint32_t)m << (2 * d));
                        c[nc++] = ch;
                    }
                }
                // one scan for both counts: records (low half), expandable records (high half)
                int total;
                const int pos = block_exclusive_scan(nc | (nl << 16), warp_sums, &total);
                for (int q = 0; q < nc; ++q)
                    nxt[outbase + (pos & 0xffff) + q] = c[q];
                outbase += total & 0xffff;
                nonleaf += total >> 16;
            }
            fmin = warp_min_int(fmin);
            if ((threadIdx.x & 31) == 0)
                atomicMin(&s_fmin, fmin);
            for (int d2 = 16; d2; d2 >>= 1)
                internal += __shfl_xor_sync(FULL, internal, d2);
            if ((threadIdx.x & 31) == 0)
                atomicAdd(&s_internal, internal);
            __syncthreads();
            cur = nxt;
            cnt = outbase;
            expandable = nonleaf;
            ++depth;
        }
        if (cur != A) {
            for (int j = threadIdx.x; j < cnt; j += blockDim.x)
                A[j] = cur[j];
        }
        if (threadIdx.x == 0) {
            a.count[k] = cnt;
            a.cnt.split_nodes[inst] = s_internal;
            a.cnt.fnext_off[inst] = s_fmin;
            if (a.fuse.jump)
                for (int m = 0; m < FUSE_K; ++m)
                    a.fuse.low[(size_t)inst * FUSE_K + m] = m < J ? s_low[m] : 0ull;
            // nodes the search may still pop in this iteration within the
            // budget (counted iterations only; path recovery is not budgeted)
            const unsigned long long budget = a.desc->node_budget;
            const unsigned long long used = st.cum_nodes + s_internal;
            a.cnt.budget_left[inst] = (budget == 0 || st.mode != MODE_COUNT) ? ~0ull
                                                                             : (budget > used ? budget - used : 0ull);
        }
    }
    if (!last_block_done<W>((unsigned *)&ctrl->done_blocks, &s_last))
        return;
    // last block: frontier offsets, then open the first pass of the step
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    const unsigned *act = ctrl->cur ? a.act1 : a.act0;
    for (int base = 0; base < n_active; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const int v = j < n_active ? __ldcg(&a.count[j]) : 0;
        int total;
        const int pos = block_exclusive_scan(v, warp_sums, &total);
        if (j < n_active)
            a.offset[j] = s_carry + pos;
        if (j < n_active && a.slice && v > 0) {
            // the frontier numbering of this iteration, kept while it runs
            a.fbase[act[j]] = s_carry + pos;
            a.fcount[act[j]] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            s_carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctrl->done_blocks = 0;
        // the first pass reads the frontiers, then the carried open nodes
        const int carried = a.slice ? ctrl->n_carry : 0;
        ctrl->n_front = s_carry;
        ctrl->n_in = s_carry + carried;
        ctrl->head = 0;
        ctrl->out_count = 0;
        ctrl->exited = 0;
        ctrl->qi = carried ? ctrl->carry_q : 0;
        ctrl->n_carry = 0;
        ctrl->step_t0 = global_ns();
        ctrl->first_pass = 1;
        ctrl->passes_step = 0;
        ctrl->t_start = ~0ull;
        ctrl->t_end = 0;
        ctrl->done_warps = 0;
        ctrl->records_total += (unsigned long long)s_carry;
        __threadfence();
        if (a.graph)
            cudaGraphSetConditional(a.h_pass, 1u);
    }
}

// End of a search pass (run by the search kernel's last warp): the records
// handed back become the next pass's input; the pass loop ends when nothing
// was handed back.
template <int W>
__device__ void end_of_pass(const Dev<W> &a)
{
    Ctrl *c = a.ctrl;
    c->passes_step += 1;
    c->passes_total += 1;
    if (c->t_end > c->t_start)
        c->search_ns += c->t_end - c->t_start;
    c->t_start = ~0ull;
    c->t_end = 0;
    c->done_warps = 0;
    c->first_pass = 0;
    c->max_out = max(c->max_out, c->out_count);
    if (c->passes_step >= MAX_PASSES_PER_STEP)
        c->err |= ERR_INTERNAL;
    bool again = c->out_count > 0 && c->err == 0;
    if (again && slice_over(a)) {
        // serving: the step's time slice is over; the open nodes wait in the
        // output queue and the next step continues their iterations
        c->n_carry = c->out_count;
        c->carry_q = c->qi ^ 1;
        again = false;
    }
    c->pass_again = again ? 1 : 0;
    if (again) {
        c->n_in = c->out_count;
        c->handed_back_total += (unsigned long long)c->out_count;
        c->head = 0;
        c->out_count = 0;
        c->exited = 0;
        c->qi ^= 1;
    }
    __threadfence();
    if (a.graph)
        cudaGraphSetConditional(a.h_pass, again ? 1u : 0u);
}

// ---------------------------------------------------------------------
// Advance: per problem, close the iteration (Algorithm 1's driver). The
// last block closes the step: the problems still active form the next one.
// ---------------------------------------------------------------------
// go: the smallest origin of a goal-bearing record; shift: how far the
// search limit of the step was above st.limit (fused iterations), which the
// record's slack is reduced by.
template <int W>
__device__ bool take_goal_record(const Dev<W> &a, const CallDesc &dsc, int k, unsigned inst, InstState<W> &st,
                                 unsigned go, int shift)
{
    const int base = a.slice ? a.fbase[inst] : a.offset[k];
    const int cnt = a.slice ? a.fcount[inst] : a.count[k];
    const int local = (int)go - base;
    if (go == 0xffffffffu || local < 0 || local >= cnt)
        return false;
    const Rec<W> r = a.scratch[region_of(a, k, inst) + local];
    const int d = (int)m_hi(r.meta);
    // every step must descend, and a goal can only sit at depth == limit
    if (st.path_len + d > st.limit || (st.mode == MODE_PATH && d == 0))
        return false;
    if (r.b == goal_board<W>() && st.path_len + d != st.limit)
        return false;
    for (int j = 0; j < d; ++j)
        dsc.out_moves[(size_t)inst * Geo<W>::MAXLEN + st.path_len + j] = (uint8_t)((r.pm >> (2 * j)) & 3u);
    st.path_len += d;
    if (st.path_len == st.limit) {
        if (r.b != goal_board<W>())
            return false;
        st.mode = MODE_DONE;
        st.status = 0;
    } else {
        const int slack = m_slack(r.meta) - shift;
        if (slack < 0)
            return false;
        st.mode = MODE_PATH;
        st.root = r.b;
        st.root_meta = m_make(m_blank(r.meta), m_last(r.meta), (uint32_t)slack);
        st.target = (uint32_t)max(2, a.tune.target_path);
    }
    return true;
}

template <int W>
__global__ void k_advance(const Dev<W> a)
{
    __shared__ int s_last;
    Ctrl *ctrl = a.ctrl;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_active = ctrl->n_active;
    if (k < n_active && ctrl->err == 0) {
        const CallDesc dsc = *a.desc;
        const unsigned inst = (ctrl->cur ? a.act1 : a.act0)[k];
        unsigned *next_active = ctrl->cur ? a.act0 : a.act1;
        if (a.slice && a.carry[inst]) {
            // its iteration continues in the next step
            next_active[atomicAdd(&ctrl->n_next, 1)] = inst;
            goto advanced;
        }
        {
        InstState<W> st = a.state[inst];
        const unsigned long long total = a.cnt.split_nodes[inst] + a.cnt.search_nodes[inst];
        const unsigned long long goals = a.cnt.goals[inst];
        if (st.mode == MODE_COUNT && ((a.cnt.aborted[inst] & ABORT_BUDGET) ||
                                      (dsc.node_budget && st.cum_nodes + total > dsc.node_budget))) {
            // the budget ran out inside this iteration: only the completed
            // iterations are reported
            st.mode = MODE_DONE;
            st.status = 4;  // BPIDA_EBUDGET
        } else if (st.mode == MODE_COUNT) {
            // the step's iterations: limits st.limit + 2j, j = 0..J (J = 0:
            // one iteration); the first with a goal ends the count
            const int J = a.fuse.jump ? st.jump : 0;
            const size_t fk = (size_t)inst * FUSE_K;
            int jg = -1;
            unsigned long long gj = goals;
            if (J == 0) {
                if (goals > 0)
                    jg = 0;
            } else {
                for (int j = 0; j <= J; ++j) {
                    const unsigned long long g = a.fuse.goals[fk + j];
                    if (g) {
                        jg = j;
                        gj = g;
                        break;
                    }
                }
            }
            const int last = jg >= 0 ? jg : J;
            // iteration j leaves out the popped nodes whose slack is below 2(J - j)
            unsigned long long excl = 0;
            for (int m = 0; m < J; ++m)
                excl += a.fuse.low[fk + m];
            unsigned long long cnt_last = 0;
            for (int j = 0; j <= last; ++j) {
                cnt_last = total - excl;
                dsc.out_nodes[(size_t)inst * Geo<W>::MAXIT + st.it + j] = cnt_last;
                st.cum_nodes += cnt_last;
                if (J - j - 1 >= 0)
                    excl -= a.fuse.low[fk + J - j - 1];
            }
            st.rows = st.it + last + 1;
            if (jg >= 0) {
                st.it += jg;
                st.limit += 2 * jg;
                st.length = st.limit;
                st.solutions = gj;
                const unsigned go = J ? a.fuse.origin[fk + jg] : a.cnt.goal_origin[inst];
                st.jump = 0;
                if (a.fuse.jump)
                    a.fuse.jump[inst] = 0;
                if (!take_goal_record<W>(a, dsc, k, inst, st, go, 2 * (J - jg))) {
                    st.mode = MODE_DONE;
                    st.status = 8;  // BPIDA_EINTERNAL
                    atomicOr(&ctrl->err, ERR_INTERNAL);
                }
            } else {
                st.it += J;
                st.limit += 2 * J;
                const int off = a.cnt.fnext_off[inst];
                if (off == INT_MAX || off <= 0) {
                    st.mode = MODE_DONE;
                    st.status = 8;
                    atomicOr(&ctrl->err, ERR_INTERNAL);
                } else if (st.it + 1 >= Geo<W>::MAXIT || st.limit + off > Geo<W>::MAXLEN) {
                    st.mode = MODE_DONE;
                    st.status = 7;  // BPIDA_ELIMIT
                } else {
                    st.limit += off;
                    st.it += 1;
                    st.root = st.start;
                    const unsigned long long g = (unsigned long long)a.tune.growth;
                    // fuse the next iterations while the top one is predicted small
                    int Jn = 0;
                    unsigned long long pred = cnt_last * g;
                    const unsigned long long cap = a.fuse.max_nodes / (unsigned long long)max(1, n_active);
                    if (a.fuse.jump)
                        while (Jn < FUSE_MAX && pred * g <= cap && st.it + Jn + 1 < Geo<W>::MAXIT &&
                               st.limit + 2 * (Jn + 1) <= Geo<W>::MAXLEN) {
                            pred *= g;
                            ++Jn;
                        }
                    st.jump = Jn;
                    if (a.fuse.jump)
                        a.fuse.jump[inst] = Jn;
                    st.root_meta =
                        m_make(m_blank(st.start_meta), LAST_NONE, (uint32_t)(st.limit + 2 * Jn - st.h0));
                    unsigned long long want = pred / (unsigned long long)a.tune.nodes_per_record;
                    want = want < 1ull ? 1ull : want;
                    want = want > (unsigned long long)a.tune.target_cap ? (unsigned long long)a.tune.target_cap : want;
                    st.target = (uint32_t)want;
                }
            }
        } else if (st.mode == MODE_PATH) {
            if (goals == 0 || !take_goal_record<W>(a, dsc, k, inst, st, a.cnt.goal_origin[inst], 0)) {
                st.mode = MODE_DONE;
                st.status = 8;
                atomicOr(&ctrl->err, ERR_INTERNAL);
            }
        }
        a.state[inst] = st;
        if (st.mode != MODE_DONE) {
            const int j = atomicAdd(&ctrl->n_next, 1);
            next_active[j] = inst;
        } else if (a.done_list) {
            a.done_list[atomicAdd(&ctrl->n_done, 1)] = inst;
        }
        }
    advanced:;
    }
    if (!last_block_done<W>((unsigned *)&ctrl->done_blocks, &s_last))
        return;
    if (threadIdx.x == 0) {
        Ctrl *c = ctrl;
        c->done_blocks = 0;
        c->n_active = *(volatile int *)&c->n_next;
        c->n_next = 0;
        c->cur ^= 1;
        c->steps += 1;
        if (c->steps >= MAX_STEPS)
            c->err |= ERR_INTERNAL;
        c->step_again = (c->n_active > 0 && *(volatile int *)&c->err == 0) ? 1 : 0;
        __threadfence();
        if (a.graph)
            cudaGraphSetConditional(a.h_step, (unsigned)c->step_again);
    }
}

// ---------------------------------------------------------------------
// Call set-up / init / finalize
// ---------------------------------------------------------------------
// Writes the call's arguments and clears the control block.
static __global__ void k_set_desc(CallDesc d, CallDesc *dst, Ctrl *ctrl)
{
    *dst = d;
    Ctrl z;
    memset(&z, 0, sizeof z);
    z.t_start = ~0ull;
    *ctrl = z;
}

// Validates board b (permutation, parity class, h0 <= max length) and sets
// up instance i: state, zeroed output rows. Returns true when the instance
// is to be searched.
template <int W, bool PDB = false>
__device__ bool init_instance(const Dev<W> &a, const CallDesc &dsc, int i, typename Geo<W>::B b)
{
    typedef typename Geo<W>::B B;
    constexpr int N = Geo<W>::N, BITS = Geo<W>::BITS;
    for (int j = 0; j < Geo<W>::MAXLEN; ++j)
        dsc.out_moves[(size_t)i * Geo<W>::MAXLEN + j] = 0;
    for (int j = 0; j < Geo<W>::MAXIT; ++j)
        dsc.out_nodes[(size_t)i * Geo<W>::MAXIT + j] = 0ull;
    InstState<W> st;
    st.start = b;
    st.root = b;
    st.it = 0;
    st.rows = 0;
    st.path_len = 0;
    st.length = -1;
    st.cum_nodes = 0;
    st.solutions = 0;
    st.target = 1;
    st.jump = 0;
    // permutation check, blank, Manhattan distance, parity class
    uint32_t seen = 0;
    int blank = -1, h = 0, inv = 0;
    bool ok = true;
    unsigned tiles[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        const unsigned t = tile_at<W>(b, p);
        tiles[p] = t;
        if (t >= (unsigned)N || (seen >> t) & 1u)
            ok = false;
        else
            seen |= 1u << t;
        if (t == 0)
            blank = p;
        else
            h += abs(p / W - (int)t / W) + abs(p % W - (int)t % W);
    }
    if constexpr (W != 4) {
        // bits above the last position must be clear
        if ((b >> (BITS * N)) != (B)0)
            ok = false;
    }
    if (ok) {
        for (int x = 0; x < N; ++x)
            for (int y = x + 1; y < N; ++y)
                if (tiles[x] && tiles[y] && tiles[x] > tiles[y])
                    ++inv;
        const int parity = (W & 1) ? (inv & 1) : ((inv + blank / W) & 1);
        ok = parity == 0;
    }
    if constexpr (PDB) {
        if (ok)
            h = pdb_h(a.pdb, *a.pdb.info, pdb_inverse<W>(b, *a.pdb.info), nullptr);
    }
    st.start_meta = 0;
    st.root_meta = 0;
    st.h0 = ok ? h : -1;
    st.limit = st.h0;
    st.mode = MODE_DONE;
    if (!ok) {
        st.status = 1;  // BPIDA_EINVAL
    } else if (h > Geo<W>::MAXLEN) {
        st.status = 7;  // BPIDA_ELIMIT
    } else {
        st.start_meta = m_make((uint32_t)blank, LAST_NONE, 0);
        st.root_meta = st.start_meta;
        st.mode = MODE_COUNT;
        st.status = 0;
        if (a.fuse.jump) {
            // the first iterations are tiny: fuse as many as the budget allows
            const unsigned long long g = (unsigned long long)a.tune.growth;
            const unsigned long long cap = a.fuse.max_nodes / (unsigned long long)max(1, dsc.n);
            unsigned long long pred = g;
            int J = 0;
            while (J < FUSE_MAX && pred * g <= cap && J + 1 < Geo<W>::MAXIT && h + 2 * (J + 1) <= Geo<W>::MAXLEN) {
                pred *= g;
                ++J;
            }
            st.jump = J;
            st.root_meta = m_make((uint32_t)blank, LAST_NONE, (uint32_t)(2 * J));
            unsigned long long want = pred / (unsigned long long)a.tune.nodes_per_record;
            want = want < 1ull ? 1ull : want;
            want = want > (unsigned long long)a.tune.target_cap ? (unsigned long long)a.tune.target_cap : want;
            st.target = (uint32_t)want;
        }
    }
    if (a.fuse.jump)
        a.fuse.jump[i] = st.jump;
    a.state[i] = st;
    return st.mode == MODE_COUNT;
}

template <int W>
__device__ __forceinline__ typename Geo<W>::B load_board(const uint64_t *boards, size_t i)
{
    typedef typename Geo<W>::B B;
    if constexpr (W <= 4)
        return (B)boards[i];
    else
        return (B)boards[2 * i] | ((B)boards[2 * i + 1] << 64);
}

template <int W, bool PDB = false>
__global__ void k_init(const Dev<W> a)
{
    __shared__ int s_last;
    const CallDesc dsc = *a.desc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < dsc.n) {
        if (init_instance<W, PDB>(a, dsc, i, load_board<W>(dsc.boards, i))) {
            const int j = atomicAdd(&a.ctrl->n_active, 1);
            a.act0[j] = (unsigned)i;
        }
    }
    if (!last_block_done<W>((unsigned *)&a.ctrl->done_blocks, &s_last))
        return;
    if (threadIdx.x == 0) {
        a.ctrl->done_blocks = 0;
        __threadfence();
        if (a.graph)
            cudaGraphSetConditional(a.h_step, *(volatile int *)&a.ctrl->n_active > 0 ? 1u : 0u);
    }
}

// Serving: admit new requests into free slots (slot[j] gets boards[j]) and
// append the searchable ones to the current active list; the rest finish
// at once (done list).
template <int W>
__global__ void k_admit(const Dev<W> a, const unsigned *slot, const uint64_t *boards, int count)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count)
        return;
    const CallDesc dsc = *a.desc;
    const unsigned i = slot[j];
    if (a.carry)
        a.carry[i] = 0;
    if (init_instance<W>(a, dsc, (int)i, load_board<W>(boards, (size_t)j))) {
        const int k = atomicAdd(&a.ctrl->n_active, 1);
        (a.ctrl->cur ? a.act1 : a.act0)[k] = i;
    } else {
        a.done_list[atomicAdd(&a.ctrl->n_done, 1)] = i;
    }
}

// Serving: marks the instances whose open nodes were carried over at the end
// of a step's time slice (they neither advance now nor split next step).
template <int W>
__global__ void k_carry_mark(const Dev<W> a)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const Ctrl *c = a.ctrl;
    if (j >= c->n_carry)
        return;
    const Rec<W> *q = c->carry_q ? a.q1 : a.q0;
    a.carry[q[j].inst] = 1u;
}

template <int W>
__global__ void k_finalize(const Dev<W> a)
{
    const CallDesc dsc = *a.desc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dsc.n)
        return;
    const int err = a.ctrl->err;
    const int abort_status = (err & ERR_QUEUE) ? 2 : 8;  // BPIDA_ENOMEM or BPIDA_EINTERNAL
    const InstState<W> st = a.state[i];
    const bool solved = st.mode == MODE_DONE && st.status == 0;
    dsc.out_len[i] = solved ? st.length : -1;
    if (dsc.out_iters)
        dsc.out_iters[i] = st.rows;
    if (dsc.out_status)
        dsc.out_status[i] = st.mode == MODE_DONE ? st.status : abort_status;
    if (dsc.out_solutions)
        dsc.out_solutions[i] = solved ? st.solutions : 0ull;
}

}  // namespace bp
