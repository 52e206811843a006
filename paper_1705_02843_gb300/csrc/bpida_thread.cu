// Thread-parallel IDA*: the three thread-based configurations that the paper
// measures before proposing BPIDA* (Section 4 and its appendix on
// thread-based parallel IDA*, Algorithm "Parallel IDA*"), kept as ablations.
// Every thread runs its own sequential f-limited depth-first search over the
// subtrees of the root nodes assigned to it:
//
//   PSimple    every iteration builds a root set of about one node per thread
//              and gives each thread one root; no load balancing.
//   PStaticLB  the root set is kept across iterations. After an iteration,
//              every root whose subtree took more nodes than the per-thread
//              average is split into at least load / average nodes (each
//              inheriting an equal share of its load as the estimate), and
//              the roots are assigned to threads in generation order so that
//              each thread receives about the average estimated load
//              (UpdateRootSet).
//   PFullLB    PStaticLB plus dynamic load balancing inside a block: when the
//              idle fraction of a block's threads passes the trigger, idle
//              threads take the shallowest untried branches of busy threads
//              of the same block through shared memory (DynamicLoadBalance).
//
// The same root-set machinery also runs the paper's BPIDA* with its own
// static load balancing (Section 5, as an ablation): the search units are
// warps (a block is one warp), each running Algorithm 1's BPDFS over its
// roots (8 nodes per parallelPop, lane i applying action i mod 4, pushes at
// ballot-reserved slots of a stack shared by the warp), and a root's load is
// the number of repetitions of BPDFS's loop it took instead of its node
// count. There is no dynamic load balancing.
//
// Root sets are built as the paper's CreateRootSet does, by an A*-style
// expansion from the start (smallest f first), without duplicate detection:
// a node is replaced in place by its children (every move but the inverse of
// the last one), goals are never expanded, and expansion stops once the set
// holds the wanted number of nodes. The set therefore does not depend on the
// limit, and PSimple builds it once. The Manhattan distance is consistent
// (h changes by exactly 1 per move), so f never decreases along a path and
// sequential IDA* at limit L pops a node exactly when its f <= L: the nodes
// expanded while building or splitting are kept as a histogram by f, and
// every iteration counts those with f <= L and takes those with f > L into
// the next limit. Node counts, lengths and solution counts therefore equal
// sequential IDA*'s. The load balance of each iteration (the largest
// per-thread node count over the mean over all threads) is recorded.
#include "bpida_thread.h"
#include "bpida_device.cuh"

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

namespace bp {
namespace tp {

constexpr int TPB = 128;     // threads per search block
constexpr int PFX = 32;      // moves a root record can carry (2 bits each)
constexpr int K_CHECK = 64;  // PFullLB: search steps between balancing checks
constexpr int HF = 128;      // f values of the expanded-node histogram (f = g + h < PFX + 60)

// A root: 24 bytes.
struct Root {
    uint64_t b;     // board (4 bits per position)
    uint64_t pm;    // moves from the start, 2 bits each, first lowest
    uint8_t blank;  // blank position
    uint8_t g;      // depth (= number of moves in pm)
    uint8_t last;   // last move, 4 = none
    uint8_t h;      // Manhattan distance
    uint32_t pad;
};

struct Ctrl {
    uint64_t start;          // start board
    int valid;               // a permutation in the goal's parity class
    int h0, blank0;
    int R;                   // roots in the set
    int fmin_off;            // smallest f - limit over pruned nodes (INT_MAX: none)
    int pad;
    unsigned long long hist[HF];  // nodes expanded by every build and update so far, by f
    unsigned long long nodes;     // nodes popped by the search threads in this iteration
    unsigned long long maxload;   // largest per-thread count in this iteration
    unsigned long long goals;     // goal nodes popped in this iteration
    unsigned long long goal_key;  // (root index << 32) | thread of the recorded goal path
    unsigned long long balances;  // PFullLB balancing operations
    unsigned long long steals;    // PFullLB branches given to idle threads
    unsigned long long reps;      // BPIDA*: repetitions of BPDFS's loop in this iteration
    int err;                      // BPIDA*: a warp's overflow stack was full
    int pad2;
    unsigned long long tot[4];    // totals of the last scans
};

// Every buffer of one solve, passed by value to the kernels.
template <int W> struct Args {
    Ctrl *ctrl;
    Root *A, *B;                      // root sets (A: current)
    unsigned long long *load;         // per root of A: nodes popped in its subtree
    unsigned long long *est;          // per root of A: load estimate
    unsigned long long *P;            // exclusive prefix sums of est
    unsigned long long *want;         // per root: split target (0 = not split)
    unsigned long long *soff;         // per root: offset of its split region
    unsigned long long *hpos;         // per root: index among the split roots
    unsigned long long *cntv;         // per split root: roots it became
    unsigned long long *npos;         // per root: offset in the new set
    unsigned *heavy;                  // indices of the roots to split
    unsigned long long *bsum;         // scan block sums
    Root *scratch;                    // split regions
    uint8_t *path;                    // per thread: the first goal path it found
    unsigned char *ovf;               // BPIDA*: per warp, an overflow stack in global memory
    uint8_t *out_moves;               // row of the current instance
    unsigned long long *out_nodes;    // row of the current instance
    int T;                            // search threads
    MoveLut<W> lut;
};

// ---------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------
template <int W> __host__ __device__ __forceinline__ unsigned legal_mask(int p)
{
    const int r = p / W, c = p % W;
    return (r > 0 ? 1u : 0u) | (c > 0 ? 2u : 0u) | (c < W - 1 ? 4u : 0u) | (r < W - 1 ? 8u : 0u);
}

template <int W> __device__ __forceinline__ int md(unsigned t, int p)
{
    const int tr = (int)t / W, tc = (int)t % W, pr = p / W, pc = p % W;
    return abs(tr - pr) + abs(tc - pc);
}

__device__ __forceinline__ unsigned excl_of(unsigned last) { return last < 4u ? (1u << (3u - last)) : 0u; }

template <int W> __device__ __forceinline__ bool expandable(const Root &r)
{
    return r.h > 0 && r.g < PFX;
}

template <int W> __device__ __forceinline__ int n_children(const Root &r)
{
    return __popc(legal_mask<W>(r.blank) & ~excl_of(r.last));
}

template <int W> __device__ __forceinline__ Root child_of(const Root &r, int m)
{
    const int p = r.blank, np = p + move_off<W>(m);
    const unsigned t = tile_at<W>(r.b, np);
    Root c;
    c.b = r.b ^ ((uint64_t)t << (4 * p)) ^ ((uint64_t)t << (4 * np));
    c.pm = r.pm | ((uint64_t)m << (2 * r.g));
    c.blank = (uint8_t)np;
    c.g = (uint8_t)(r.g + 1);
    c.last = (uint8_t)m;
    c.h = (uint8_t)((int)r.h - md<W>(t, np) + md<W>(t, p));
    c.pad = 0;
    return c;
}

// Block-wide exclusive scan of 64-bit values (blockDim a multiple of 32).
__device__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *ws, unsigned long long *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, x, d);
        if (lane >= d)
            x += y;
    }
    if (lane == 31)
        ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < nw ? ws[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, s, d);
            if (lane >= d)
                s += y;
        }
        if (lane < nw)
            ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = (wid > 0 ? ws[wid - 1] : 0ull) + x - v;
    *total = ws[nw - 1];
    __syncthreads();
    return before;
}

// ---------------------------------------------------------------------
// Exclusive scan of n 64-bit values (three kernels), total to *total.
// ---------------------------------------------------------------------
constexpr int SC_T = 512, SC_V = 8, SC_B = SC_T * SC_V;

__global__ void __launch_bounds__(SC_T) k_scan_a(const unsigned long long *in, unsigned long long *out, int n,
                                                 unsigned long long *bsum)
{
    __shared__ unsigned long long ws[32];
    const size_t base = (size_t)blockIdx.x * SC_B + (size_t)threadIdx.x * SC_V;
    unsigned long long v[SC_V], s = 0;
#pragma unroll
    for (int k = 0; k < SC_V; ++k) {
        v[k] = base + k < (size_t)n ? in[base + k] : 0ull;
        s += v[k];
    }
    unsigned long long tot;
    unsigned long long x = block_scan_u64(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < SC_V; ++k) {
        if (base + k < (size_t)n)
            out[base + k] = x;
        x += v[k];
    }
    if (threadIdx.x == 0)
        bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_b(unsigned long long *bsum, int nb, unsigned long long *total)
{
    __shared__ unsigned long long ws[32];
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long x = block_scan_u64(v, ws, &tot);
        if (i < nb)
            bsum[i] = carry + x;
        carry += tot;
    }
    if (threadIdx.x == 0)
        *total = carry;
}

__global__ void k_scan_c(unsigned long long *out, int n, const unsigned long long *bsum)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (size_t)n)
        out[i] += bsum[i / SC_B];
}

cudaError_t scan(const unsigned long long *in, unsigned long long *out, int n, unsigned long long *bsum,
                 unsigned long long *total, cudaStream_t st)
{
    const int nb = (n + SC_B - 1) / SC_B;
    if (nb > 0)
        k_scan_a<<<nb, SC_T, 0, st>>>(in, out, n, bsum);
    k_scan_b<<<1, 1024, 0, st>>>(bsum, nb, total);
    if (nb > 0)
        k_scan_c<<<(n + 1023) / 1024, 1024, 0, st>>>(out, n, bsum);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Root-set construction
// ---------------------------------------------------------------------
// Block-wide. Replaces, in place and in order, nodes of the list `cur` (cnt
// nodes) by their children until the list holds at least `target` nodes or
// nothing in it is expandable: each step takes the smallest f among the
// expandable nodes and expands, in list order, the nodes with that f, up to
// the first prefix of the list whose expansion reaches the target. `alt` is
// the other buffer; both hold at least target + 4 nodes. Expanded nodes are
// added to the histogram by f. Returns the buffer that holds the result.
template <int W>
__device__ Root *partial_expand(Root *cur, Root *alt, int &cnt, int target, unsigned long long *hist,
                                unsigned long long *ws)
{
    __shared__ int s_k, s_f;
    __shared__ unsigned s_exp;
    while (cnt < target) {
        const unsigned long long need = (unsigned long long)(target - cnt);
        if (threadIdx.x == 0) {
            s_k = -1;
            s_f = INT_MAX;
            s_exp = 0;
        }
        __syncthreads();
        // the smallest f among the expandable nodes
        int fm = INT_MAX;
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const Root r = cur[j];
            if (expandable<W>(r))
                fm = min(fm, (int)r.g + (int)r.h);
        }
        fm = warp_min_int(fm);
        if ((threadIdx.x & 31) == 0 && fm != INT_MAX)
            atomicMin(&s_f, fm);
        __syncthreads();
        const int fs = s_f;
        if (fs == INT_MAX)
            break;
        // the shortest prefix whose expansion reaches the target
        unsigned long long run = 0;
        for (int base = 0; base < cnt; base += blockDim.x) {
            const int j = base + threadIdx.x;
            unsigned long long gain = 0;
            if (j < cnt) {
                const Root r = cur[j];
                if (expandable<W>(r) && (int)r.g + (int)r.h == fs)
                    gain = (unsigned long long)(n_children<W>(r) - 1);
            }
            unsigned long long tot;
            const unsigned long long ex = block_scan_u64(gain, ws, &tot);
            if (j < cnt && run + ex < need && run + ex + gain >= need)
                s_k = j + 1;
            run += tot;
            __syncthreads();
            if (s_k >= 0)
                break;
        }
        const int k = s_k >= 0 ? s_k : cnt;
        __syncthreads();
        // write the new list
        unsigned long long run2 = 0;
        for (int base = 0; base < cnt; base += blockDim.x) {
            const int j = base + threadIdx.x;
            Root r;
            r.b = 0;
            r.pm = 0;
            r.blank = r.g = r.last = r.h = 0;
            r.pad = 0;
            bool ex_j = false;
            unsigned long long gain = 0;
            if (j < cnt) {
                r = cur[j];
                ex_j = j < k && expandable<W>(r) && (int)r.g + (int)r.h == fs;
                if (ex_j)
                    gain = (unsigned long long)(n_children<W>(r) - 1);
            }
            unsigned long long tot;
            const unsigned long long ex = block_scan_u64(gain, ws, &tot);
            if (j < cnt) {
                size_t pos = (size_t)j + run2 + ex;
                if (ex_j) {
                    const unsigned allow = legal_mask<W>(r.blank) & ~excl_of(r.last);
                    for (int m = 0; m < 4; ++m)
                        if ((allow >> m) & 1u)
                            alt[pos++] = child_of<W>(r, m);
                    atomicAdd(&s_exp, 1u);
                } else {
                    alt[pos] = r;
                }
            }
            run2 += tot;
        }
        cnt += (int)run2;
        Root *t = cur;
        cur = alt;
        alt = t;
        __syncthreads();
        if (threadIdx.x == 0 && s_exp)
            atomicAdd(&hist[fs], (unsigned long long)s_exp);
    }
    return cur;
}

// The root set of every variant's first iteration (PSimple keeps it): about
// T roots from the start. One block.
template <int W> __global__ void __launch_bounds__(1024) k_build(const Args<W> a, int target)
{
    __shared__ unsigned long long ws[32];
    Ctrl *c = a.ctrl;
    if (threadIdx.x == 0) {
        Root r;
        r.b = c->start;
        r.pm = 0;
        r.blank = (uint8_t)c->blank0;
        r.g = 0;
        r.last = 4;
        r.h = (uint8_t)c->h0;
        r.pad = 0;
        a.A[0] = r;
    }
    __syncthreads();
    int cnt = 1;
    Root *res = partial_expand<W>(a.A, a.B, cnt, target, c->hist, ws);
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        if (res != a.A)
            a.A[j] = res[j];
        a.est[j] = 1ull;
    }
    if (threadIdx.x == 0)
        c->R = cnt;
}

// PStaticLB update, step 1: which roots to split, and into how many. A root
// is split when its load exceeds the per-thread average prev / T (prev: the
// nodes the threads popped in the previous iteration), into at least
// ceil(load / average) roots.
template <int W> __global__ void k_mark(const Args<W> a, int R, unsigned long long prev)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R)
        return;
    const unsigned long long ld = a.load[j];
    const unsigned long long T = (unsigned long long)a.T;
    const bool heavy = prev > 0 && ld * T > prev && expandable<W>(a.A[j]);
    const unsigned long long m = heavy ? (ld * T + prev - 1) / prev : 0ull;
    a.want[j] = m;
    a.soff[j] = heavy ? 2 * (m + 4) : 0ull;
    a.hpos[j] = heavy ? 1ull : 0ull;
}

template <int W> __global__ void k_heavy_index(const Args<W> a, int R)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < R && a.want[j])
        a.heavy[a.hpos[j]] = (unsigned)j;
}

// Step 2: one block per root to split, expanded smallest f first in the
// root's own scratch region (two halves of want + 4 nodes).
template <int W> __global__ void __launch_bounds__(TPB) k_split_heavy(const Args<W> a)
{
    __shared__ unsigned long long ws[32];
    const unsigned j = a.heavy[blockIdx.x];
    const int m = (int)a.want[j];
    Root *cur = a.scratch + a.soff[j];
    Root *alt = cur + (m + 4);
    if (threadIdx.x == 0)
        cur[0] = a.A[j];
    __syncthreads();
    int cnt = 1;
    Root *res = partial_expand<W>(cur, alt, cnt, m, a.ctrl->hist, ws);
    if (res != cur)
        for (int q = threadIdx.x; q < cnt; q += blockDim.x)
            cur[q] = res[q];
    if (threadIdx.x == 0)
        a.cntv[j] = (unsigned long long)cnt;
}

template <int W> __global__ void k_counts(const Args<W> a, int R)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < R)
        a.npos[j] = a.want[j] ? a.cntv[j] : 1ull;
}

// Step 3: the new set (in A's order, each split root replaced by its
// roots) with the load estimates for the coming iteration.
template <int W> __global__ void k_compose(const Args<W> a, int R)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R)
        return;
    const unsigned long long ld = a.load[j];
    const size_t o = a.npos[j];
    if (a.want[j]) {
        const unsigned long long n = a.cntv[j];
        const unsigned long long e = ld > n ? (ld + n - 1) / n : 1ull;
        const Root *src = a.scratch + a.soff[j];
        for (unsigned long long q = 0; q < n; ++q) {
            a.B[o + q] = src[q];
            a.est[o + q] = e;
        }
    } else {
        a.B[o] = a.A[j];
        a.est[o] = ld > 1ull ? ld : 1ull;
    }
}

// The set kept as it is: estimates from the measured loads.
template <int W> __global__ void k_est_from_load(const Args<W> a, int R)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < R)
        a.est[j] = a.load[j] > 1ull ? a.load[j] : 1ull;
}

// ---------------------------------------------------------------------
// Search
// ---------------------------------------------------------------------
struct Offer {
    uint64_t b, rpm;
    uint32_t sh;
    int s, mask, k, rg, donor;
    unsigned root;
    int pad;
};

// First root of thread t: the roots are cut into T consecutive runs of about
// equal estimated load (exclusive prefix sums P, total E).
__device__ __forceinline__ int first_root(const unsigned long long *P, int R, unsigned long long E, int T, int t)
{
    if (t >= T)
        return R;
    const unsigned long long want = (unsigned long long)t * E;
    int lo = 0, hi = R;  // first j with P[j] * T >= t * E
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] * (unsigned long long)T >= want)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

template <int W, bool DLB> struct Searcher {
    typedef typename Geo<W>::B B;
    static constexpr int BITS = Geo<W>::BITS, MAXD = Geo<W>::MAXLEN;

    const Args<W> &a;
    const unsigned char *lut;
    uint8_t *stk;  // level-major: level k of thread i at stk[k * TPB + i]
    uint8_t *col;  // this thread's column
    int L, j, jend;
    unsigned gt;
    // depth-first state of the current piece of work
    B b;
    uint32_t sh;
    int s, d, base;
    bool have;
    unsigned root;
    int rg;
    uint64_t rpm;
    unsigned long long nodes, seg, goals;
    bool recorded;
    int fmin;

    __device__ Searcher(const Args<W> &args, const unsigned char *lut_, uint8_t *stk_, int L_, int j0, int j1)
        : a(args), lut(lut_), stk(stk_), col(stk_ + threadIdx.x), L(L_), j(j0), jend(j1),
          gt(blockIdx.x * TPB + threadIdx.x), b(0), sh(0), s(0), d(0), base(0), have(false), root(0), rg(0),
          rpm(0), nodes(0), seg(0), goals(0), recorded(false), fmin(INT_MAX)
    {
    }

    __device__ __forceinline__ bool idle() const { return !have && j >= jend; }

    __device__ void record_goal()
    {
        ++goals;
        if (recorded)
            return;
        recorded = true;
        uint8_t *pb = a.path + (size_t)gt * MAXD;
        int n = 0;
        for (int k = 0; k < rg; ++k)
            pb[n++] = (uint8_t)((rpm >> (2 * k)) & 3u);
        for (int k = 1; k <= d; ++k)
            pb[n++] = (uint8_t)(col[k * TPB] >> 4);
        atomicMin(&a.ctrl->goal_key, ((unsigned long long)root << 32) | gt);
    }

    // Undoes move m (the move that made the node at the current level) on
    // (bb, shh, ss).
    __device__ __forceinline__ void undo(B &bb, uint32_t &shh, int &ss, int m) const
    {
        const uint32_t sh_p = (uint32_t)((int)shh - BITS * move_off<W>(m));
        const unsigned t = BoardOps<W>::tile(bb, sh_p);
        const bool away = away_bit<W>(lut_row_sh<W>(lut, sh_p), m, t);
        bb = BoardOps<W>::flip(bb, t * move_mul<W>(m), m < 2 ? shh : sh_p);
        shh = sh_p;
        ss += away ? 2 : 0;
    }

    // One step: take a root, try a move, or go back up one level.
    __device__ __forceinline__ void step()
    {
        if (!have) {
            if (j < jend) {
                const Root r = a.A[j];
                const int f = (int)r.g + (int)r.h;
                if (f > L) {
                    fmin = min(fmin, f - L);
                } else {
                    ++nodes;
                    root = (unsigned)j;
                    rg = r.g;
                    rpm = r.pm;
                    d = 0;
                    if (r.h == 0) {
                        record_goal();
                        atomicAdd(&a.load[j], 1ull);
                    } else {
                        b = (B)r.b;
                        sh = (uint32_t)(BITS * r.blank);
                        s = L - f;
                        base = 0;
                        seg = nodes - 1;
                        col[0] = (uint8_t)(legal_mask<W>(r.blank) & ~excl_of(r.last));
                        have = true;
                    }
                }
                ++j;
            }
            return;
        }
        const uint32_t e = col[d * TPB];
        const uint32_t mask = e & 15u;
        if (mask) {
            const int m = __ffs(mask) - 1;
            col[d * TPB] = (uint8_t)(e & ~(1u << m));
            const uint32_t sh_np = (uint32_t)((int)sh + BITS * move_off<W>(m));
            const unsigned t = BoardOps<W>::tile(b, sh_np);
            const bool away = away_bit<W>(lut_row_sh<W>(lut, sh), m, t);
            if (away && s < 2) {
                fmin = min(fmin, 2 - s);  // f of the child is limit + 2 - s
                return;
            }
            b = BoardOps<W>::flip(b, t * move_mul<W>(m), m < 2 ? sh_np : sh);
            sh = sh_np;
            s -= away ? 2 : 0;
            ++d;
            ++nodes;
            if (b == goal_board<W>()) {
                col[d * TPB] = (uint8_t)(m << 4);  // goals are not expanded
                record_goal();
            } else {
                const unsigned p = sh / BITS;
                col[d * TPB] = (uint8_t)((m << 4) | (legal_mask<W>((int)p) & ~(1u << (3 - m))));
            }
        } else if (d == base) {
            have = false;
            atomicAdd(&a.load[root], nodes - seg);
        } else {
            undo(b, sh, s, (int)(e >> 4));
            --d;
        }
    }

    // PFullLB: idle threads take the shallowest untried branches of busy
    // threads of the block (block-wide; every thread calls it).
    __device__ void balance(Offer *offers, int *warp_sums)
    {
        int kmin = -1;
        if (have)
            for (int k = base; k < d; ++k)
                if (col[k * TPB] & 15u) {
                    kmin = k;
                    break;
                }
        const bool donor = kmin >= 0;
        const bool idl = idle();
        int total;
        const int pos = block_exclusive_scan((idl ? 1 : 0) | (donor ? 1 << 16 : 0), warp_sums, &total);
        const int npair = min(total & 0xffff, total >> 16);
        const int irank = pos & 0xffff, drank = pos >> 16;
        if (donor && drank < npair) {
            B b2 = b;
            uint32_t sh2 = sh;
            int s2 = s;
            for (int k = d; k > kmin; --k)
                undo(b2, sh2, s2, (int)(col[k * TPB] >> 4));
            Offer o;
            o.b = (uint64_t)b2;
            o.rpm = rpm;
            o.sh = sh2;
            o.s = s2;
            o.mask = (int)(col[kmin * TPB] & 15u);
            o.k = kmin;
            o.rg = rg;
            o.donor = (int)threadIdx.x;
            o.root = root;
            o.pad = 0;
            offers[drank] = o;
            col[kmin * TPB] = (uint8_t)(col[kmin * TPB] & 0xF0u);
        }
        __syncthreads();
        if (idl && irank < npair) {
            const Offer o = offers[irank];
            const uint8_t *dc = stk + o.donor;
            for (int k = 1; k <= o.k; ++k)
                col[k * TPB] = (uint8_t)(dc[k * TPB] & 0xF0u);
            col[o.k * TPB] = (uint8_t)((o.k > 0 ? (col[o.k * TPB] & 0xF0u) : 0u) | (unsigned)o.mask);
            b = (B)o.b;
            sh = o.sh;
            s = o.s;
            d = base = o.k;
            root = o.root;
            rg = o.rg;
            rpm = o.rpm;
            seg = nodes;
            have = true;
        }
        __syncthreads();
        if (threadIdx.x == 0 && npair > 0)
            atomicAdd(&a.ctrl->steals, (unsigned long long)npair);
    }
};

template <int W, bool DLB> constexpr size_t search_smem()
{
    return SharedLut<W>::BYTES + (size_t)(Geo<W>::MAXLEN + 1) * TPB +
           (DLB ? ((size_t)TPB * sizeof(Offer) + 16) : 0);
}

template <int W, bool DLB>
__global__ void __launch_bounds__(TPB) k_search_tp(const Args<W> a, int L, int R, unsigned long long E)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int warp_sums[32];
    __shared__ long long s_last_end, s_cost;
    __shared__ int s_go;
    unsigned char *lut = smem;
    uint8_t *stk = smem + SharedLut<W>::BYTES;
    SharedLut<W>::load(lut, a.lut);
    if (threadIdx.x == 0) {
        s_last_end = clock64();
        s_cost = 0;
        s_go = 0;
    }
    __syncthreads();
    const int t = blockIdx.x * TPB + threadIdx.x;
    Searcher<W, DLB> S(a, lut, stk, L, first_root(a.P, R, E, a.T, t), first_root(a.P, R, E, a.T, t + 1));
    if (!DLB) {
        while (!S.idle())
            S.step();
    } else {
        Offer *offers =
            (Offer *)(((uintptr_t)(stk + (size_t)(Geo<W>::MAXLEN + 1) * TPB) + 15) & ~(uintptr_t)15);
        for (;;) {
            for (int k = 0; k < K_CHECK; ++k)
                S.step();
            const int n_idle = __syncthreads_count(S.idle());
            if (n_idle == (int)blockDim.x)
                break;
            if (n_idle == 0)
                continue;
            // Trigger: balance once the idle fraction reaches c / (c + t),
            // c = duration of the previous balancing, t = time since it
            // ended, and no sooner than c / 2 after it.
            if (threadIdx.x == 0) {
                const long long tt = clock64() - s_last_end, c = s_cost;
                s_go = (2 * tt >= c) && ((long long)n_idle * (c + tt) >= (long long)blockDim.x * c);
            }
            __syncthreads();
            if (s_go) {
                const long long t0 = clock64();
                S.balance(offers, warp_sums);
                if (threadIdx.x == 0) {
                    s_last_end = clock64();
                    s_cost = s_last_end - t0;
                    atomicAdd(&a.ctrl->balances, 1ull);
                }
            }
            __syncthreads();
        }
    }
    // per-warp reduction of the counters
    unsigned long long n = S.nodes, mx = S.nodes, g = S.goals;
    int fm = S.fmin;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        n += __shfl_xor_sync(FULL, n, o);
        mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        g += __shfl_xor_sync(FULL, g, o);
        fm = min(fm, __shfl_xor_sync(FULL, fm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (n)
            atomicAdd(&a.ctrl->nodes, n);
        atomicMax(&a.ctrl->maxload, mx);
        if (g)
            atomicAdd(&a.ctrl->goals, g);
        if (fm != INT_MAX)
            atomicMin(&a.ctrl->fmin_off, fm);
    }
}

// ---------------------------------------------------------------------
// The paper's BPIDA* search (Algorithm 1): one warp per unit
// ---------------------------------------------------------------------
constexpr int BPW_S = 512;        // shared-memory stack entries per warp
constexpr int BPW_OVF = 2048;      // overflow stack entries per warp (global memory)

constexpr size_t bpw_smem() { return SharedLut<4>::BYTES + (size_t)BPW_S * WarpStack<4>::ENTRY_BYTES; }

// Warp u searches the roots [first_root(u), first_root(u + 1)) one after
// another. For each root with f <= L, BPDFS: the stack starts with the root;
// every repetition pops the top n <= 8 nodes (parallelPop), lanes 4q..4q+3
// take node q, goal-test it (a goal is counted and not expanded), and lane
// 4q + m applies move m; a child with f <= L is pushed at a ballot-reserved
// slot (atomicPut), the others lower f_next. The repetitions a root took are
// its load for the next iteration's rebalancing. When the shared stack
// cannot take a repetition's children, its oldest half moves to the warp's
// overflow stack in global memory, and comes back when the shared stack has
// drained; a full overflow stack sets err (the call fails, nothing hangs).
template <int W>
__global__ void __launch_bounds__(32) k_search_bpw(const Args<W> a, int L, int R, unsigned long long E)
{
    typedef typename Geo<W>::B B;
    constexpr int BITS = Geo<W>::BITS, S = BPW_S;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *lut = smem;
    SharedLut<W>::load(lut, a.lut);
    __syncthreads();
    WarpStack<W> stk, ovf;
    stk.init(smem + SharedLut<W>::BYTES, S);
    ovf.init(a.ovf + (size_t)blockIdx.x * BPW_OVF * WarpStack<W>::ENTRY_BYTES, BPW_OVF);
    const int lane = threadIdx.x & 31, q = lane >> 2, m = lane & 3;
    const unsigned lt = (1u << lane) - 1u;
    const B GOAL = goal_board<W>();
    const int j0 = first_root(a.P, R, E, a.T, blockIdx.x), j1 = first_root(a.P, R, E, a.T, blockIdx.x + 1);
    unsigned long long nodes = 0, goals = 0, reps_all = 0;
    int fmin = INT_MAX;
    unsigned goal_root = 0xffffffffu;
    bool failed = false;
    for (int j = j0; j < j1 && !failed; ++j) {
        const Root r = a.A[j];
        const int f = (int)r.g + (int)r.h;
        if (f > L) {
            fmin = min(fmin, f - L);
            continue;
        }
        if (lane == 0)
            stk.put(0, (B)r.b, sm_from_rec<W>(m_make(r.blank, r.last, (uint32_t)(L - f))), 0u);
        __syncwarp();
        int top = 1, ovn = 0;
        unsigned long long reps = 0;
        while (top > 0 || ovn > 0) {
            if (top == 0) {
                // refill from the overflow stack (its most recent entries)
                const int k = min(ovn, S / 2);
                for (int i = lane; i < k; i += 32) {
                    B bb;
                    uint32_t mm, oo;
                    ovf.get(ovn - k + i, bb, mm, oo);
                    stk.put(i, bb, mm, oo);
                }
                ovn -= k;
                top = k;
                __syncwarp();
            }
            const int n = min(8, top);
            if (top + 3 * n > S) {
                // room for 4n children: the oldest entries go to global memory
                const int k = min(top - n, S / 2);
                if (ovn + k > BPW_OVF) {
                    failed = true;
                    break;
                }
                for (int i = lane; i < k; i += 32) {
                    B bb;
                    uint32_t mm, oo;
                    stk.get(i, bb, mm, oo);
                    ovf.put(ovn + i, bb, mm, oo);
                }
                ovn += k;
                __syncwarp();
                for (int i0 = 0; i0 < top - k; i0 += 32) {
                    const int i = i0 + lane;
                    const bool ok = i < top - k;
                    B bb = 0;
                    uint32_t mm = 0, oo = 0;
                    if (ok)
                        stk.get(k + i, bb, mm, oo);
                    __syncwarp();
                    if (ok)
                        stk.put(i, bb, mm, oo);
                    __syncwarp();
                }
                top -= k;
            }
            // parallelPop: the top n nodes, four lanes per node
            const bool act = q < n;
            B b = 0;
            uint32_t mt = 0, org = 0;
            if (act)
                stk.get(top - n + q, b, mt, org);
            top -= n;
            nodes += (unsigned long long)n;
            ++reps;
            __syncwarp();
            const bool goal = act && b == GOAL;
            const unsigned gm = __ballot_sync(FULL, goal && m == 0);
            if (gm) {
                goals += (unsigned long long)__popc(gm);
                goal_root = min(goal_root, (unsigned)j);
            }
            const uint32_t sh_p = mt & 127u;
            const int s = (int)((mt >> 11) & 255u);
            // the (threadID mod #actions)th action
            const bool legal = act && !goal && ((LegalMoves<W>::at_sh(sh_p) & ~((mt >> 7) & 15u)) >> m & 1u);
            const uint32_t sh_np = sh_p + (uint32_t)(BITS * move_off<W>(m));
            const unsigned t = BoardOps<W>::tile(b, sh_np);
            const bool away = away_bit<W>(lut_row_sh<W>(lut, sh_p), m, t);
            const bool push = legal && !(away && s < 2);
            if (legal && away && s < 2)
                fmin = min(fmin, 2 - s);
            const B child = BoardOps<W>::flip(b, t * move_mul<W>(m), (m < 2) ? sh_np : sh_p);
            const uint32_t cm = (sh_np + (mt & (255u << 11)) + ((1u << (3 - m)) << 7)) - (away ? (2u << 11) : 0u);
            const unsigned pm = __ballot_sync(FULL, push);
            if (push)
                stk.put(top + __popc(pm & lt), child, cm, 0u);
            top += __popc(pm);
            __syncwarp();
        }
        if (lane == 0)
            a.load[j] = reps;
        reps_all += reps;
    }
    fmin = warp_min_int(fmin);
    if (lane == 0) {
        if (nodes)
            atomicAdd(&a.ctrl->nodes, nodes);
        atomicMax(&a.ctrl->maxload, nodes);
        if (goals)
            atomicAdd(&a.ctrl->goals, goals);
        if (fmin != INT_MAX)
            atomicMin(&a.ctrl->fmin_off, fmin);
        if (reps_all)
            atomicAdd(&a.ctrl->reps, reps_all);
        if (goal_root != 0xffffffffu)
            atomicMin(&a.ctrl->goal_key, (unsigned long long)goal_root << 32);
        if (failed)
            atomicOr(&a.ctrl->err, 1);
    }
}

// ---------------------------------------------------------------------
// Per-instance set-up and results
// ---------------------------------------------------------------------
template <int W> __global__ void k_init(const Args<W> a, const uint64_t *boards, int i)
{
    constexpr int N = W * W;
    for (int k = threadIdx.x; k < Geo<W>::MAXLEN; k += blockDim.x)
        a.out_moves[k] = 0;
    for (int k = threadIdx.x; k < Geo<W>::MAXIT; k += blockDim.x)
        a.out_nodes[k] = 0ull;
    if (threadIdx.x != 0)
        return;
    const uint64_t b = boards[i];
    Ctrl *c = a.ctrl;
    uint32_t seen = 0;
    int blank = -1, h = 0, inv = 0;
    bool ok = true;
    unsigned tiles[N];
    for (int p = 0; p < N; ++p) {
        const unsigned t = tile_at<W>(b, p);
        tiles[p] = t;
        if (t >= (unsigned)N || ((seen >> t) & 1u))
            ok = false;
        else
            seen |= 1u << t;
        if (t == 0)
            blank = p;
        else
            h += md<W>(t, p);
    }
    if (W != 4 && (b >> (4 * N)) != 0)
        ok = false;
    if (ok) {
        for (int x = 0; x < N; ++x)
            for (int y = x + 1; y < N; ++y)
                if (tiles[x] && tiles[y] && tiles[x] > tiles[y])
                    ++inv;
        ok = ((W & 1) ? (inv & 1) : ((inv + blank / W) & 1)) == 0;
    }
    Ctrl z;
    memset(&z, 0, sizeof z);
    z.start = b;
    z.valid = ok ? 1 : 0;
    z.h0 = ok ? h : -1;
    z.blank0 = blank;
    z.fmin_off = INT_MAX;
    z.goal_key = ~0ull;
    *c = z;
}

template <int W> __global__ void k_reset_iter(const Args<W> a)
{
    Ctrl *c = a.ctrl;
    c->nodes = 0;
    c->maxload = 0;
    c->goals = 0;
    c->goal_key = ~0ull;
    c->fmin_off = INT_MAX;
    c->reps = 0;
}

template <int W> __global__ void k_close(const Args<W> a, int it, unsigned long long internal)
{
    a.out_nodes[it] = internal + a.ctrl->nodes;
}

// sols: the solution count, or ~0 for the goals the search counted
template <int W>
__global__ void k_finish(const Args<W> a, int i, int status, int length, int iters, int *out_len, int *out_iters,
                         int *out_status, uint64_t *out_solutions, unsigned long long sols)
{
    const bool ok = status == BPIDA_OK;
    if (ok) {
        const unsigned t = (unsigned)(a.ctrl->goal_key & 0xffffffffull);
        const uint8_t *pb = a.path + (size_t)t * Geo<W>::MAXLEN;
        for (int k = threadIdx.x; k < length; k += blockDim.x)
            a.out_moves[k] = pb[k];
    }
    if (threadIdx.x == 0) {
        out_len[i] = ok ? length : -1;
        if (out_iters)
            out_iters[i] = iters;
        if (out_status)
            out_status[i] = status;
        if (out_solutions)
            out_solutions[i] = ok ? (sols != ~0ull ? sols : a.ctrl->goals) : 0ull;
    }
}

// ---------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------
struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

struct Workspace {
    Buf ctrl, A, B, load, est, P, want, soff, hpos, cntv, npos, heavy, bsum, scratch, path, ovf;
    Ctrl *h_ctrl = nullptr;
    cudaError_t ensure(Buf &b, size_t bytes)
    {
        bytes = std::max<size_t>(bytes, 256);
        if (b.n >= bytes)
            return cudaSuccess;
        if (b.p)
            cudaFree(b.p);
        b.p = nullptr;
        b.n = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e == cudaSuccess)
            b.n = bytes;
        return e;
    }
    void release()
    {
        Buf *all[] = {&ctrl, &A, &B, &load, &est, &P, &want, &soff, &hpos, &cntv, &npos, &heavy, &bsum, &scratch,
                      &path, &ovf};
        for (Buf *b : all) {
            if (b->p)
                cudaFree(b->p);
            b->p = nullptr;
            b->n = 0;
        }
        if (h_ctrl)
            cudaFreeHost(h_ctrl);
        h_ctrl = nullptr;
    }
};

std::vector<Workspace *> g_ws;

#define TK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            std::fprintf(stderr, "bpida (thread-parallel): %s failed: %s\n", #x, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? BPIDA_ENOMEM : BPIDA_ECUDA;                  \
        }                                                                                         \
    } while (0)

struct Totals {
    double ratio_prev = 0.0, ratio_last = 0.0;
    unsigned long long roots = 0, balances = 0, steals = 0;
};

template <int W, bool DLB, bool BPW>
bpida_status solve_one(const Settings &cfg, Workspace &ws, Args<W> a, const uint64_t *boards, int i, int grid,
                       int Rcap, size_t Scap, int *out_len, int *out_iters, int *out_status,
                       uint64_t *out_solutions, cudaStream_t st, Totals &tot, bpida_stats *stats)
{
    constexpr int MAXLEN = Geo<W>::MAXLEN, MAXIT = Geo<W>::MAXIT;
    a.out_moves += (size_t)i * MAXLEN;
    a.out_nodes += (size_t)i * MAXIT;
    const int T = a.T;
    const int th = 256;
    Ctrl &hc = *ws.h_ctrl;
    auto fetch = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(ws.h_ctrl, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
    };
    auto finish = [&](int status, int length, int iters, unsigned long long sols = ~0ull) -> bpida_status {
        k_finish<W><<<1, 128, 0, st>>>(a, i, status, length, iters, out_len, out_iters, out_status, out_solutions,
                                      sols);
        TK(cudaGetLastError());
        return (bpida_status)status;
    };

    k_init<W><<<1, 128, 0, st>>>(a, boards, i);
    TK(cudaGetLastError());
    TK(fetch());
    stats->launches += 1;
    if (!hc.valid)
        return finish(BPIDA_EINVAL, -1, 0);
    if (hc.h0 > MAXLEN)
        return finish(BPIDA_ELIMIT, -1, 0);

    int L = hc.h0, it = 0, R = 0;
    unsigned long long prev = 0;
    std::vector<double> ratio;
    for (;;) {
        k_reset_iter<W><<<1, 1, 0, st>>>(a);
        TK(cudaGetLastError());
        stats->launches += 1;
        if (it == 0) {
            // CreateRootSet (PSimple keeps this set in every iteration)
            k_build<W><<<1, 1024, 0, st>>>(a, std::min(T, Rcap - 4));
            TK(cudaGetLastError());
            TK(fetch());
            R = hc.R;
            stats->launches += 1;
        } else if (cfg.variant != PSIMPLE) {
            // UpdateRootSet: split the roots that took more than the average
            const int gb = (R + th - 1) / th;
            k_mark<W><<<gb, th, 0, st>>>(a, R, prev);
            TK(cudaGetLastError());
            TK(scan(a.soff, a.soff, R, a.bsum, &a.ctrl->tot[0], st));
            TK(scan(a.hpos, a.hpos, R, a.bsum, &a.ctrl->tot[1], st));
            TK(fetch());
            const unsigned long long S_tot = hc.tot[0], H = hc.tot[1];
            stats->launches += 7;
            // fewer than T roots can take more than the average, so the
            // split regions (2 * (want + 4) nodes each) always fit in Scap;
            // the set itself may reach Rcap, and is then kept as it is
            const bool fits = H > 0 && S_tot <= Scap && (unsigned long long)R + S_tot / 2 <= (unsigned long long)Rcap;
            if (fits) {
                k_heavy_index<W><<<gb, th, 0, st>>>(a, R);
                k_split_heavy<W><<<(unsigned)H, TPB, 0, st>>>(a);
                k_counts<W><<<gb, th, 0, st>>>(a, R);
                TK(cudaGetLastError());
                TK(scan(a.npos, a.npos, R, a.bsum, &a.ctrl->tot[2], st));
                TK(fetch());
                const int Rn = (int)hc.tot[2];
                k_compose<W><<<gb, th, 0, st>>>(a, R);
                TK(cudaGetLastError());
                std::swap(a.A, a.B);
                R = Rn;
                stats->launches += 7;
            } else {
                k_est_from_load<W><<<gb, th, 0, st>>>(a, R);
                TK(cudaGetLastError());
                stats->launches += 1;
            }
        }
        // expanded nodes popped at this limit, and the smallest f above it
        unsigned long long internal = 0;
        int hist_off = INT_MAX;
        for (int f = 0; f < HF; ++f) {
            if (f <= L)
                internal += hc.hist[f];
            else if (hc.hist[f] && hist_off == INT_MAX)
                hist_off = f - L;
        }
        // assignment: prefix sums of the estimates
        TK(scan(a.est, a.P, R, a.bsum, &a.ctrl->tot[3], st));
        TK(cudaMemsetAsync(a.load, 0, sizeof(unsigned long long) * (size_t)R, st));
        TK(fetch());
        const unsigned long long E = hc.tot[3];
        if (BPW)
            k_search_bpw<W><<<grid, 32, bpw_smem(), st>>>(a, L, R, E);
        else
            k_search_tp<W, DLB><<<grid, TPB, search_smem<W, DLB>(), st>>>(a, L, R, E);
        TK(cudaGetLastError());
        k_close<W><<<1, 1, 0, st>>>(a, it, internal);
        TK(cudaGetLastError());
        TK(fetch());
        stats->launches += 6;
        stats->passes += 1;
        stats->search_nodes += hc.nodes;
        const double avg = (double)hc.nodes / (double)T;
        ratio.push_back(avg > 0.0 ? (double)hc.maxload / avg : 0.0);
        tot.balances = hc.balances;
        tot.steals = hc.steals;
        tot.roots = (unsigned long long)R;
        tot.ratio_last = ratio.back();
        tot.ratio_prev = ratio.size() >= 2 ? ratio[ratio.size() - 2] : ratio.back();
        stats->steps += 1;
        if (BPW && hc.err)
            return finish(BPIDA_ENOMEM, -1, it + 1);
        if (hc.goals > 0 && BPW) {
            // the path: the roots are in the order of their move sequences
            // (CreateRootSet and the splits replace a node by its children in
            // move order), so the first root with a goal, searched depth
            // first in move order by one thread, gives the lexicographically
            // first optimal solution (its counts are not used)
            const unsigned long long sols = hc.goals;
            const size_t gr = (size_t)(hc.goal_key >> 32);
            Args<W> one = a;
            one.A = a.B;
            one.T = TPB;
            TK(cudaMemcpyAsync(one.A, a.A + gr, sizeof(Root), cudaMemcpyDeviceToDevice, st));
            TK(cudaMemsetAsync(a.P, 0, sizeof(unsigned long long), st));
            k_reset_iter<W><<<1, 1, 0, st>>>(a);
            k_search_tp<W, false><<<1, TPB, search_smem<W, false>(), st>>>(one, L, 1, 1ull);
            TK(cudaGetLastError());
            stats->launches += 2;
            return finish(BPIDA_OK, L, it + 1, sols);
        }
        if (hc.goals > 0)
            return finish(BPIDA_OK, L, it + 1);
        const int off = std::min(hc.fmin_off, hist_off);
        if (off == INT_MAX || off <= 0)
            return finish(BPIDA_EINTERNAL, -1, it + 1);
        if (it + 1 >= MAXIT || L + off > MAXLEN)
            return finish(BPIDA_ELIMIT, -1, it + 1);
        L += off;
        ++it;
        prev = BPW ? hc.reps : hc.nodes;
    }
}

template <int W, bool DLB, bool BPW>
bpida_status solve_wd(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                      uint64_t *out_nodes, int *out_iters, int *out_status, uint64_t *out_solutions, cudaStream_t st,
                      bpida_stats *stats)
{
    int dev = 0, sms = 0;
    TK(cudaGetDevice(&dev));
    TK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if ((int)g_ws.size() <= dev)
        g_ws.resize(dev + 1, nullptr);
    if (!g_ws[dev])
        g_ws[dev] = new Workspace();
    Workspace &ws = *g_ws[dev];

    // search units: threads, or warps (BPIDA*: a block is one warp)
    const int unit_threads = BPW ? 32 : TPB;
    const size_t smem = BPW ? bpw_smem() : search_smem<W, DLB>();
    static int bpsm = 0;  // per (W, DLB, BPW) instantiation
    if (bpsm == 0) {
        if (BPW)
            TK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_search_bpw<W>, 32, smem));
        else
            TK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_search_tp<W, DLB>, TPB, smem));
    }
    if (bpsm < 1)
        return BPIDA_EINVAL;
    const int grid = cfg.threads > 0 ? (BPW ? cfg.threads : (cfg.threads + TPB - 1) / TPB) : sms * bpsm;
    const int T = BPW ? grid : grid * TPB;
    const long long rcap = (long long)(cfg.variant == PSIMPLE ? 2 : 32) * T + 4096;
    if (rcap > (1ll << 30))
        return BPIDA_ENOMEM;
    const int Rcap = (int)rcap;
    const size_t Scap = (size_t)12 * T + 4096;
    const size_t u64 = sizeof(unsigned long long);

    TK(ws.ensure(ws.ctrl, sizeof(Ctrl)));
    TK(ws.ensure(ws.A, sizeof(Root) * (size_t)Rcap));
    TK(ws.ensure(ws.B, sizeof(Root) * (size_t)Rcap));
    TK(ws.ensure(ws.load, u64 * Rcap));
    TK(ws.ensure(ws.est, u64 * Rcap));
    TK(ws.ensure(ws.P, u64 * Rcap));
    TK(ws.ensure(ws.want, u64 * Rcap));
    TK(ws.ensure(ws.soff, u64 * Rcap));
    TK(ws.ensure(ws.hpos, u64 * Rcap));
    TK(ws.ensure(ws.cntv, u64 * Rcap));
    TK(ws.ensure(ws.npos, u64 * Rcap));
    TK(ws.ensure(ws.heavy, sizeof(unsigned) * (size_t)Rcap));
    TK(ws.ensure(ws.bsum, u64 * ((size_t)Rcap / SC_B + 2)));
    TK(ws.ensure(ws.scratch, sizeof(Root) * Scap));
    TK(ws.ensure(ws.path, (size_t)std::max(T, TPB) * Geo<W>::MAXLEN));
    if (BPW)
        TK(ws.ensure(ws.ovf, (size_t)T * BPW_OVF * WarpStack<W>::ENTRY_BYTES));
    if (!ws.h_ctrl)
        TK(cudaMallocHost((void **)&ws.h_ctrl, sizeof(Ctrl)));

    Args<W> a;
    std::memset(&a, 0, sizeof a);
    a.ctrl = (Ctrl *)ws.ctrl.p;
    a.A = (Root *)ws.A.p;
    a.B = (Root *)ws.B.p;
    a.load = (unsigned long long *)ws.load.p;
    a.est = (unsigned long long *)ws.est.p;
    a.P = (unsigned long long *)ws.P.p;
    a.want = (unsigned long long *)ws.want.p;
    a.soff = (unsigned long long *)ws.soff.p;
    a.hpos = (unsigned long long *)ws.hpos.p;
    a.cntv = (unsigned long long *)ws.cntv.p;
    a.npos = (unsigned long long *)ws.npos.p;
    a.heavy = (unsigned *)ws.heavy.p;
    a.bsum = (unsigned long long *)ws.bsum.p;
    a.scratch = (Root *)ws.scratch.p;
    a.path = (uint8_t *)ws.path.p;
    a.ovf = (unsigned char *)ws.ovf.p;
    a.out_moves = out_moves;
    a.out_nodes = (unsigned long long *)out_nodes;
    a.T = T;
    a.lut = make_move_lut<W>();

    stats->grid_blocks = grid;
    stats->block_threads = unit_threads;
    stats->sm_count = sms;
    stats->tp_threads = T;
    bpida_status first = BPIDA_OK;
    Totals tot;
    unsigned long long balances = 0, steals = 0;
    for (int i = 0; i < n; ++i) {
        const bpida_status s = solve_one<W, DLB, BPW>(cfg, ws, a, boards, i, grid, Rcap, Scap, out_len, out_iters,
                                                 out_status, out_solutions, st, tot, stats);
        // per-instance outcomes (invalid board, length cap) go to out_status
        if (s == BPIDA_ECUDA || s == BPIDA_ENOMEM)
            return s;
        if (s == BPIDA_EINTERNAL)
            first = s;
        balances += tot.balances;
        steals += tot.steals;
    }
    TK(cudaStreamSynchronize(st));
    stats->lb_ratio = tot.ratio_prev;
    stats->lb_ratio_last = tot.ratio_last;
    stats->tp_roots = tot.roots;
    stats->tp_balances = balances;
    stats->tp_steals = steals;
    return first;
}

bpida_status solve(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                   uint64_t *out_nodes, int *out_iters, int *out_status, uint64_t *out_solutions, cudaStream_t st,
                   bpida_stats *stats)
{
#define TP_SOLVE(W_, DLB_, BPW_)                                                                              \
    solve_wd<W_, DLB_, BPW_>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_solutions, \
                             st, stats)
    if (cfg.variant == BPSTATIC)
        return cfg.width == 3 ? TP_SOLVE(3, false, true) : TP_SOLVE(4, false, true);
    const bool dlb = cfg.variant == PFULLLB;
    if (cfg.width == 3)
        return dlb ? TP_SOLVE(3, true, false) : TP_SOLVE(3, false, false);
    return dlb ? TP_SOLVE(4, true, false) : TP_SOLVE(4, false, false);
#undef TP_SOLVE
}

void release(int dev)
{
    if (dev < (int)g_ws.size() && g_ws[dev])
        g_ws[dev]->release();
}

}  // namespace tp
}  // namespace bp
