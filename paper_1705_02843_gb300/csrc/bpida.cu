// Host side of the GB300 Block-Parallel IDA* solver: the C ABI declared in
// include/bpida.h and the threshold loop of Algorithm 1 (BPIDA*).
//
// One solve call runs all of its instances together. Every step closes one
// f-limited iteration of every still-active instance (each at its own
// limit), or several consecutive ones searched together (fused iterations,
// calls of a few boards): k_split builds each instance's root set (its last
// block computes the frontier offsets), k_search passes consume the
// frontiers with persistent warps (another pass only when warps handed work
// back; the last block of a pass decides), and k_advance records the
// iterations' node counts and raises each limit to the smallest pruned f,
// or, once a goal was popped, walks down the first goal-bearing root to
// recover the solution path (its last block closes the step).
//
// By default the whole loop is one CUDA graph: the step loop and the pass
// loop are conditional WHILE nodes whose conditions are set on the device,
// so a call is two launches enqueued on the caller's stream (the argument
// block, then the graph) and returns without waiting: calls are
// stream-ordered and asynchronous. Each call takes a workspace of its own
// from a small per-device pool: the one last used on the same stream (the
// stream orders the two calls), else an idle one, else a new one, so calls
// on different streams run concurrently. The host-driven loop (driver = 1)
// launches the same kernels one by one and reads the control block back
// after every pass (it synchronises the stream); it is what times each
// search launch with CUDA events.
#include "bpida.h"
#include "bpida_device.cuh"
#include "bpida_pdb.h"
#include "bpida_thread.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

using namespace bp;

namespace bp {
void noalloc_forget(int dev);  // bpida_noalloc.cu
}

namespace {

thread_local bpida_stats g_stats;
thread_local int g_timing = 0;
// search launches of this thread's last host-driven call with timing on:
// CUDA-event duration (ms) and the nodes the launch popped
struct LaunchRec {
    double ms;
    uint64_t nodes;
};
thread_local std::vector<LaunchRec> g_launch_log;
std::atomic<unsigned long long> g_fuse_nodes{0};  // 0: the defaults below
std::mutex g_mu;

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
};

// W, S, warps per block, n, frontier cap, hand-back percentage, min rounds, min pass time, variant,
// fused iterations, pattern databases (their id; 0 = Manhattan distance), fused-step node cap
typedef std::tuple<int, int, int, int, int, int, int, int, int, int, unsigned long long, unsigned long long>
    PlanKey;

struct Plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned gen = 0;  // workspace generation the graph was built for
    unsigned long long last_use = 0;
    void destroy()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (graph)
            cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
};

struct Workspace {
    DevBuf state, act0, act1, ctr, scratch, count, offset, q0, q1, ctrl, desc, ovf, fuse;
    Ctrl *h_ctrl = nullptr;  // pinned copy of the control block, written at the end of each call
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t done = nullptr;         // recorded after the last call's work
    cudaStream_t last_stream = nullptr;  // stream of the last call
    bool used = false;                  // a call has been enqueued with it
    unsigned long long last_call = 0;
    unsigned gen = 1;  // bumped whenever a buffer moves
    std::map<PlanKey, Plan> plans;
    unsigned long long use_clock = 0;

    // Keeps at most MAX_PLANS instantiated graphs (least recently used go
    // first) and drops every graph built for buffers that have since moved.
    static constexpr size_t MAX_PLANS = 8;
    void trim_plans()
    {
        // a graph may still be running: wait before destroying any
        if (!plans.empty())
            wait_idle();
        for (auto it = plans.begin(); it != plans.end();) {
            if (!it->second.exec || it->second.gen != gen) {
                it->second.destroy();
                it = plans.erase(it);
            } else {
                ++it;
            }
        }
        while (plans.size() >= MAX_PLANS) {
            auto lru = plans.begin();
            for (auto it = plans.begin(); it != plans.end(); ++it)
                if (it->second.last_use < lru->second.last_use)
                    lru = it;
            lru->second.destroy();
            plans.erase(lru);
        }
    }

    // The last call's work has finished (before a buffer is freed).
    cudaError_t wait_idle()
    {
        return used && done ? cudaEventSynchronize(done) : cudaSuccess;
    }

    cudaError_t ensure(DevBuf &b, size_t bytes)
    {
        bytes = std::max<size_t>(bytes, 256);
        if (b.n >= bytes)
            return cudaSuccess;
        if (b.p) {
            const cudaError_t e = wait_idle();
            if (e != cudaSuccess)
                return e;
            cudaFree(b.p);
        }
        b.p = nullptr;
        b.n = 0;
        ++gen;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e == cudaSuccess)
            b.n = bytes;
        return e;
    }
    void release()
    {
        wait_idle();
        for (auto &kv : plans)
            kv.second.destroy();
        plans.clear();
        DevBuf *all[] = {&state, &act0, &act1, &ctr, &scratch, &count, &offset, &q0, &q1, &ctrl, &desc, &ovf,
                         &fuse};
        for (DevBuf *b : all) {
            if (b->p)
                cudaFree(b->p);
            b->p = nullptr;
            b->n = 0;
        }
        ++gen;
        if (h_ctrl)
            cudaFreeHost(h_ctrl);
        h_ctrl = nullptr;
        if (ev0)
            cudaEventDestroy(ev0);
        if (ev1)
            cudaEventDestroy(ev1);
        if (done)
            cudaEventDestroy(done);
        ev0 = ev1 = done = nullptr;
        used = false;
        last_stream = nullptr;
    }
};

// Per device, a pool of at most MAX_WORKSPACES workspaces.
constexpr size_t MAX_WORKSPACES = 4;
std::vector<std::vector<Workspace *>> g_ws;
unsigned long long g_calls = 0;

// The workspace for a call on stream st (under g_mu): the one whose last
// call was on st (the stream orders the two calls), else an idle one, else a
// new one while the pool is small, else the least recently used one, with st
// made to wait (on the device) for that workspace's last call.
Workspace *workspace_for(int dev, cudaStream_t st, cudaError_t *err)
{
    *err = cudaSuccess;
    if ((int)g_ws.size() <= dev)
        g_ws.resize(dev + 1);
    std::vector<Workspace *> &pool = g_ws[dev];
    for (Workspace *w : pool)
        if (w->used && w->last_stream == st)
            return w;
    for (Workspace *w : pool)
        if (!w->used || cudaEventQuery(w->done) == cudaSuccess)
            return w;
    cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error of this call
    if (pool.size() < MAX_WORKSPACES) {
        pool.push_back(new Workspace());
        return pool.back();
    }
    Workspace *lru = pool[0];
    for (Workspace *w : pool)
        if (w->last_call < lru->last_call)
            lru = w;
    *err = cudaStreamWaitEvent(st, lru->done, 0);
    return lru;
}

// The calling thread's last graph-driven call: its workspace, whose pinned
// control block receives the call's loop state at the end of the call, and
// the call's number (the workspace may have served a later call since).
struct LastCall {
    Workspace *ws = nullptr;
    unsigned long long call = 0;
};
thread_local LastCall g_last;

// The statistics that come from the control block of a finished call.
void fill_loop_stats(bpida_stats &s, const Ctrl &c, bool graph)
{
    s.steps = c.steps;
    s.passes = (int)c.passes_total;
    s.records = c.records_total;
    s.handed_back = c.handed_back_total;
    s.search_nodes = c.search_nodes_total;
    s.spills = c.spills;
    s.max_handed_back = c.max_out;
    s.search_ms_device = (double)c.search_ns * 1e-6;
    if (graph)  // k_set_desc, k_init, k_finalize; k_split and k_advance per step; k_search per pass
        s.launches = 3 + 2 * c.steps + (int)c.passes_total;
}

struct Settings {
    int width, count_all, split_target, wpb, S, exit_pct, min_rounds, driver, min_pass_ns, variant;
    uint64_t budget;
    const bpida_pdb *pdb;  // pattern databases, or null (Manhattan distance)
};

// A step fuses the next iterations of an instance while the highest of them
// is predicted (x tune.growth per iteration) to expand at most this many
// nodes (divided among the step's instances): the small early iterations
// share one step instead of one each. Calls with at most FUSE_MAX_N boards
// use it (their steps are few and short, so the steps saved pay); larger
// batches run the kernel without the fused counts.
// (One value for both heuristics: with pattern databases h(start) lies closer
// to the optimum, so a fused step searches thresholds above the solution
// more often, but smaller caps cost more in extra steps than they save.)
constexpr unsigned long long FUSE_NODES = 8000000ull;
constexpr int FUSE_MAX_N = 8;

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            std::fprintf(stderr, "bpida: %s failed: %s\n", #x, cudaGetErrorString(e_));          \
            return e_ == cudaErrorMemoryAllocation ? BPIDA_ENOMEM : BPIDA_ECUDA;                  \
        }                                                                                         \
    } while (0)

// Adds a kernel node; the arguments are copied into the node.
template <typename... P, typename... A>
cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep, size_t ndep,
                       void (*f)(P...), dim3 grid, dim3 block, size_t smem, A... args)
{
    void *ptrs[] = {(void *)&args...};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = (void *)f;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = ptrs;
    return cudaGraphAddKernelNode(node, g, dep, ndep, &kp);
}

cudaError_t add_while(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep, size_t ndep,
                      cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, ndep, &cp);
    if (e == cudaSuccess)
        *body = cp.conditional.phGraph_out[0];
    return e;
}

struct Geometry {
    int grid, threads, total_warps, C, tcap;
    size_t smem, Q;
    int n_cap;
    int variant;
    bool fuse;
};

// variant 0: warp per subtree group; 1: the paper's kernel; 6: block per
// subtree group (the autotuner's other mode, widths 3 and 4)
constexpr int VARIANT_BLOCK = 6;
template <int W, int S, bool PDB> void (*search_kernel(int variant, bool fuse))(const Dev<W>)
{
    if constexpr (PDB) {
        return fuse ? k_search<W, S, true, true> : k_search<W, S, false, true>;
    } else {
        if constexpr (W <= 4)
            if (variant == VARIANT_BLOCK)
                return k_search_block<W, S>;
        return variant == 1 ? k_search_paper<W, S> : fuse ? k_search<W, S, true> : k_search<W, S, false>;
    }
}

// The whole solve as one graph (k_set_desc is launched before it):
//   init -> WHILE(step){ split -> WHILE(pass){ search } -> advance } -> finalize
template <int W, int S, bool PDB>
cudaError_t build_graph(Plan &pl, Dev<W> d, const Geometry &g, const char **where)
{
    cudaGraph_t G;
    *where = "cudaGraphCreate";
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e != cudaSuccess)
        return e;
    pl.graph = G;
    cudaGraphConditionalHandle hs, hp;
    *where = "step handle";
    if ((e = cudaGraphConditionalHandleCreate(&hs, G, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return e;
    d.graph = 1;
    d.h_step = hs;
    d.h_pass = 0;
    const dim3 b128(128), bsplit(SPLIT_THREADS);
    const dim3 g_inst((g.n_cap + 127) / 128), g_prob(g.n_cap);
    cudaGraphNode_t n_init, n_step, n_fin;
    *where = "init/step/finalize nodes";
    if ((e = add_kernel(&n_init, G, nullptr, 0, k_init<W, PDB>, g_inst, b128, 0, d)) != cudaSuccess)
        return e;
    cudaGraph_t B;
    if ((e = add_while(&n_step, G, &n_init, 1, hs, &B)) != cudaSuccess)
        return e;
    if ((e = add_kernel(&n_fin, G, &n_step, 1, k_finalize<W>, g_inst, b128, 0, d)) != cudaSuccess)
        return e;

    *where = "pass handle";
    if ((e = cudaGraphConditionalHandleCreate(&hp, B, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return e;
    d.h_pass = hp;
    cudaGraphNode_t n_split, n_pass, n_adv;
    *where = "split/pass/advance nodes";
    if ((e = add_kernel(&n_split, B, nullptr, 0, k_split<W, PDB>, g_prob, bsplit, 0, d)) != cudaSuccess)
        return e;
    cudaGraph_t P;
    if ((e = add_while(&n_pass, B, &n_split, 1, hp, &P)) != cudaSuccess)
        return e;
    if ((e = add_kernel(&n_adv, B, &n_pass, 1, k_advance<W>, g_inst, b128, 0, d)) != cudaSuccess)
        return e;

    cudaGraphNode_t n_search;
    *where = "search node";
    if ((e = add_kernel(&n_search, P, nullptr, 0, search_kernel<W, S, PDB>(g.variant, g.fuse), dim3(g.grid), dim3(g.threads),
                        g.smem, d)) != cudaSuccess)
        return e;
    *where = "cudaGraphInstantiate";
    return cudaGraphInstantiate(&pl.exec, G, 0);
}

template <int W, int S, bool PDB = false>
bpida_status run(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                 uint64_t *out_nodes, int *out_iters, int *out_status, uint64_t *out_solutions, cudaStream_t st)
{
    g_launch_log.clear();
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaError_t wse = cudaSuccess;
    Workspace &ws = *workspace_for(dev, st, &wse);
    CK(wse);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    Geometry g;
    g.n_cap = n;
    g.variant = cfg.variant;
    // fused iterations: this kernel, no node budget, a call of at most
    // FUSE_MAX_N boards (in first-solution mode a fused step runs to
    // completion and only an unfused step stops at the first goal)
    const bool fuse = cfg.variant == 0 && cfg.budget == 0 && n <= FUSE_MAX_N;
    g.fuse = fuse;
    const int wpb = cfg.variant == 1 ? 1 : cfg.wpb;  // the paper's kernel: block = warp
    g.threads = wpb * 32;
    // search stack entries: 16 bytes, 24 for W = 5 and the pattern-database search
    g.smem = SearchSmem<W, PDB>::TABLES + (size_t)wpb * S * WarpStack<W, (W == 5) || PDB>::ENTRY_BYTES;
    // one kernel serves every block size (and the serving path), so its
    // dynamic shared memory limit is set once to the device's maximum; the
    // blocks per SM are looked up once per (device, block size, kernel)
    static std::map<std::tuple<int, int, int>, int> smem_limit;
    int &lim = smem_limit[std::make_tuple(dev, cfg.variant, fuse ? 1 : 0)];
    if (lim == 0) {
        // the device maximum less the kernel's static shared memory
        int optin = 0;
        cudaFuncAttributes fa;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CK(cudaFuncGetAttributes(&fa, search_kernel<W, S, PDB>(cfg.variant, fuse)));
        lim = optin - (int)fa.sharedSizeBytes;
        CK(cudaFuncSetAttribute(search_kernel<W, S, PDB>(cfg.variant, fuse), cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    }
    if (g.smem > (size_t)lim)
        return BPIDA_EINVAL;
    static std::map<std::tuple<int, int, int, int>, int> occ;
    int &bpsm = occ[std::make_tuple(dev, wpb, cfg.variant, fuse ? 1 : 0)];
    if (bpsm == 0)
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, search_kernel<W, S, PDB>(cfg.variant, fuse), g.threads, g.smem));
    if (bpsm < 1)
        return BPIDA_EINVAL;
    g.grid = sms * bpsm;
    g.total_warps = g.grid * wpb;
    g.tcap = cfg.split_target > 0 ? cfg.split_target : std::max(2, std::min(4096, (1 << 21) / std::max(n, 1)));
    g.C = 4 * g.tcap + 4;
    // per-warp overflow stacks, and the hand-back queue: every warp's shared
    // and overflow stacks plus its unfinished chunk, twice over; overflowing
    // it is detected and reported as BPIDA_ENOMEM
    const int ovf_cap = (W == 5) ? 4 * S : 0;
    g.Q = std::max({(size_t)n * g.C, (size_t)g.total_warps * (S + ovf_cap + 32) * 2, (size_t)1 << 24}) + 1024;
    if (g.Q > (size_t)INT_MAX / 2 || (size_t)n * 2 * g.C > (size_t)UINT32_MAX)
        return BPIDA_ENOMEM;

    CK(ws.ensure(ws.state, sizeof(InstState<W>) * n));
    CK(ws.ensure(ws.act0, sizeof(unsigned) * n));
    CK(ws.ensure(ws.act1, sizeof(unsigned) * n));
    CK(ws.ensure(ws.ctr, (size_t)n * (4 * sizeof(unsigned long long) + sizeof(int) + 2 * sizeof(unsigned))));
    CK(ws.ensure(ws.scratch, sizeof(Rec<W>) * (size_t)n * 2 * g.C));
    CK(ws.ensure(ws.count, sizeof(int) * n));
    CK(ws.ensure(ws.offset, sizeof(int) * n));
    CK(ws.ensure(ws.q0, sizeof(Rec<W>) * g.Q));
    CK(ws.ensure(ws.q1, sizeof(Rec<W>) * g.Q));
    CK(ws.ensure(ws.ctrl, sizeof(Ctrl)));
    CK(ws.ensure(ws.desc, sizeof(CallDesc)));
    CK(ws.ensure(ws.ovf, (size_t)g.total_warps * ovf_cap * WarpStack<W>::ENTRY_BYTES));
    if (fuse)
        CK(ws.ensure(ws.fuse, (size_t)n * (sizeof(int) + FUSE_K * (2 * sizeof(unsigned long long) + sizeof(unsigned)))));
    if (!ws.h_ctrl)
        CK(cudaMallocHost((void **)&ws.h_ctrl, sizeof(Ctrl)));
    if (!ws.ev0) {
        CK(cudaEventCreate(&ws.ev0));
        CK(cudaEventCreate(&ws.ev1));
        CK(cudaEventCreateWithFlags(&ws.done, cudaEventDisableTiming));
    }

    Dev<W> d;
    std::memset(&d, 0, sizeof d);
    d.ctrl = (Ctrl *)ws.ctrl.p;
    d.desc = (const CallDesc *)ws.desc.p;
    d.state = (InstState<W> *)ws.state.p;
    d.act0 = (unsigned *)ws.act0.p;
    d.act1 = (unsigned *)ws.act1.p;
    d.scratch = (Rec<W> *)ws.scratch.p;
    d.q0 = (Rec<W> *)ws.q0.p;
    d.q1 = (Rec<W> *)ws.q1.p;
    d.count = (int *)ws.count.p;
    d.offset = (int *)ws.offset.p;
    d.C = g.C;
    d.Q = (int)g.Q;
    d.ovf = (unsigned char *)ws.ovf.p;
    d.ovf_cap = ovf_cap;
    if (fuse) {
        char *p = (char *)ws.fuse.p;
        d.fuse.low = (unsigned long long *)p;
        p += sizeof(unsigned long long) * FUSE_K * n;
        d.fuse.goals = (unsigned long long *)p;
        p += sizeof(unsigned long long) * FUSE_K * n;
        d.fuse.origin = (unsigned *)p;
        p += sizeof(unsigned) * FUSE_K * n;
        d.fuse.jump = (int *)p;
        const unsigned long long set = g_fuse_nodes.load();
        d.fuse.max_nodes = set ? set : FUSE_NODES;
    }
    {
        char *p = (char *)ws.ctr.p;
        d.cnt.search_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        d.cnt.split_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        d.cnt.goals = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        d.cnt.budget_left = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        d.cnt.fnext_off = (int *)p;
        p += sizeof(int) * n;
        d.cnt.goal_origin = (unsigned *)p;
        p += sizeof(unsigned) * n;
        d.cnt.aborted = (unsigned *)p;
    }
    d.tune.min_rounds = cfg.min_rounds;
    d.tune.exit_threshold = std::max(1, (int)((long long)g.total_warps * cfg.exit_pct / 100));
    d.tune.nodes_per_record = 4096;
    d.tune.target_cap = g.tcap;
    d.tune.target_path = std::min(g.tcap, 4096);
    d.tune.growth = 8;
    d.tune.min_pass_ns = cfg.min_pass_ns;
    d.lut = make_move_lut<W>();
    if constexpr (PDB) {
        d.pdb.tab = cfg.pdb->tab;
        d.pdb.info = cfg.pdb->d_info;
        d.pdb.goal = cfg.pdb->goal;
        d.pdb.goal_sb = cfg.pdb->goal_sb;
    }

    CallDesc desc;
    std::memset(&desc, 0, sizeof desc);
    desc.boards = boards;
    desc.out_len = out_len;
    desc.out_moves = out_moves;
    desc.out_nodes = (unsigned long long *)out_nodes;
    desc.out_iters = out_iters;
    desc.out_status = out_status;
    desc.out_solutions = (unsigned long long *)out_solutions;
    desc.node_budget = cfg.budget;
    desc.n = n;
    desc.first_only = cfg.count_all ? 0 : 1;
    k_set_desc<<<1, 1, 0, st>>>(desc, (CallDesc *)ws.desc.p, d.ctrl);
    CK(cudaGetLastError());

    bpida_stats stats;
    std::memset(&stats, 0, sizeof stats);
    stats.grid_blocks = g.grid;
    stats.block_threads = g.threads;
    stats.sm_count = sms;

    const dim3 b128(128), bsplit(SPLIT_THREADS);
    const dim3 g_inst((n + 127) / 128);
    if (cfg.driver == 0) {
        const PlanKey key(W, S, cfg.wpb, n, g.tcap, cfg.exit_pct, cfg.min_rounds, cfg.min_pass_ns, cfg.variant,
                          fuse ? 1 : 0, PDB ? cfg.pdb->id : 0ull, fuse ? d.fuse.max_nodes : 0ull);
        auto found = ws.plans.find(key);
        if (found == ws.plans.end() || !found->second.exec || found->second.gen != ws.gen) {
            ws.trim_plans();
            Plan &pl = ws.plans[key];
            const char *where = "";
            cudaError_t e = build_graph<W, S, PDB>(pl, d, g, &where);
            if (e != cudaSuccess) {
                std::fprintf(stderr, "bpida: graph build failed at %s: %s\n", where, cudaGetErrorString(e));
                pl.destroy();
                ws.plans.erase(key);
                return BPIDA_ECUDA;
            }
            pl.gen = ws.gen;
            found = ws.plans.find(key);
        }
        Plan &pl = found->second;
        pl.last_use = ++ws.use_clock;
        CK(cudaGraphLaunch(pl.exec, st));
        // the loop state goes to the pinned copy at the end of the call;
        // bpida_get_stats reads it once the caller has synchronised
        CK(cudaMemcpyAsync(ws.h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(ws.done, st));
        ws.used = true;
        ws.last_stream = st;
        ws.last_call = ++g_calls;
        g_stats = stats;
        g_last.ws = &ws;
        g_last.call = ws.last_call;
        // problems the device finds (queue capacity, a failed internal check)
        // are reported per instance by k_finalize
        return BPIDA_OK;
    }
    // host-driven loop over the same kernels (synchronous)
    d.graph = 0;
    k_init<W, PDB><<<g_inst, b128, 0, st>>>(d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws.h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stats.launches = 2;
    unsigned long long nodes_seen = ws.h_ctrl->search_nodes_total;
    int n_active = ws.h_ctrl->n_active;
    while (n_active > 0) {
        k_split<W, PDB><<<n_active, bsplit, 0, st>>>(d);
        CK(cudaGetLastError());
        stats.launches += 1;
        for (;;) {
            if (g_timing)
                CK(cudaEventRecord(ws.ev0, st));
            search_kernel<W, S, PDB>(cfg.variant, fuse)<<<g.grid, g.threads, g.smem, st>>>(d);
            CK(cudaGetLastError());
            if (g_timing)
                CK(cudaEventRecord(ws.ev1, st));
            stats.launches += 1;
            CK(cudaMemcpyAsync(ws.h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (g_timing) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1));
                stats.search_ms += ms;
                g_launch_log.push_back({(double)ms, ws.h_ctrl->search_nodes_total - nodes_seen});
            }
            nodes_seen = ws.h_ctrl->search_nodes_total;
            if (!ws.h_ctrl->pass_again)
                break;
        }
        k_advance<W><<<(n_active + 127) / 128, b128, 0, st>>>(d);
        CK(cudaGetLastError());
        stats.launches += 1;
        CK(cudaMemcpyAsync(ws.h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        n_active = ws.h_ctrl->step_again ? ws.h_ctrl->n_active : 0;
    }
    k_finalize<W><<<g_inst, b128, 0, st>>>(d);
    CK(cudaGetLastError());
    stats.launches += 1;
    CK(cudaMemcpyAsync(ws.h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ws.done, st));
    ws.used = true;
    ws.last_stream = st;
    ws.last_call = ++g_calls;
    CK(cudaStreamSynchronize(st));
    fill_loop_stats(stats, *ws.h_ctrl, false);
    g_stats = stats;
    g_last.ws = nullptr;
    const Ctrl &c = *ws.h_ctrl;
    if (c.err & ERR_QUEUE)
        return BPIDA_ENOMEM;
    if (c.err)
        return BPIDA_EINTERNAL;
    return BPIDA_OK;
}

template <int W>
bpida_status run_w(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                   uint64_t *out_nodes, int *out_iters, int *out_status, uint64_t *out_sol, cudaStream_t st)
{
    if (cfg.pdb) {
        // pattern databases: 8- and 15-puzzle, stacks of 256, 384 or 512 entries
        if constexpr (W <= 4) {
            if (cfg.S == 256)
                return run<W, 256, true>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status,
                                         out_sol, st);
            if (cfg.S == 384)
                return run<W, 384, true>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status,
                                         out_sol, st);
            if (cfg.S == 512)
                return run<W, 512, true>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status,
                                         out_sol, st);
        }
        return BPIDA_EINVAL;
    }
    switch (cfg.S) {
    case 256: return run<W, 256>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    case 384: return run<W, 384>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    case 480: return run<W, 480>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    case 768: return run<W, 768>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    case 1024: return run<W, 1024>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    default: return run<W, 512>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, out_sol, st);
    }
}

}  // namespace

extern "C" {

int bpida_max_len(int width)
{
    switch (width) {
    case 3: return Geo<3>::MAXLEN;
    case 4: return Geo<4>::MAXLEN;
    case 5: return Geo<5>::MAXLEN;
    }
    return 0;
}

int bpida_max_iters(int width)
{
    switch (width) {
    case 3: return Geo<3>::MAXIT;
    case 4: return Geo<4>::MAXIT;
    case 5: return Geo<5>::MAXIT;
    }
    return 0;
}

}  // extern "C"

namespace {

// Reads a config (null: defaults) and checks what the host can check.
bpida_status parse_settings(const bpida_config *cfg_in, int n, Settings &cfg)
{
    cfg.width = (cfg_in && cfg_in->width) ? cfg_in->width : 4;
    cfg.count_all = cfg_in ? cfg_in->count_all : 1;
    cfg.split_target = cfg_in ? cfg_in->split_target : 0;
    cfg.wpb = (cfg_in && cfg_in->warps_per_block > 0) ? cfg_in->warps_per_block : 4;
    // more resident warps outweigh the extra stack spills: 15-puzzle 384
    // entries (eight 4-warp search blocks per SM), 24-puzzle 384 (24-byte
    // entries); 8-puzzle 512
    cfg.S = (cfg_in && cfg_in->stack_entries > 0) ? cfg_in->stack_entries
                                                  : (cfg.width == 3 ? 512 : 384);
    cfg.exit_pct = (cfg_in && cfg_in->exit_fraction_pct > 0) ? cfg_in->exit_fraction_pct : 10;
    cfg.min_rounds = (cfg_in && cfg_in->min_rounds > 0) ? cfg_in->min_rounds : 64;
    cfg.driver = cfg_in ? cfg_in->driver : 0;
    cfg.variant = cfg_in ? cfg_in->variant : 0;
    cfg.min_pass_ns = (cfg_in && cfg_in->min_pass_us != 0) ? (cfg_in->min_pass_us < 0 ? 0 : cfg_in->min_pass_us * 1000)
                                                             : 10000;
    cfg.budget = cfg_in ? cfg_in->node_budget : 0;
    cfg.pdb = nullptr;
    if (cfg.width < 3 || cfg.width > 5 || n < 0)
        return BPIDA_EINVAL;
    if (cfg.S != 256 && cfg.S != 384 && cfg.S != 480 && cfg.S != 512 && cfg.S != 768 && cfg.S != 1024)
        return BPIDA_EINVAL;
    if (cfg.wpb < 1 || cfg.wpb > 32 || cfg.exit_pct > 100 || cfg.split_target < 0 || cfg.split_target > (1 << 20))
        return BPIDA_EINVAL;
    if (cfg.driver != 0 && cfg.driver != 1)
        return BPIDA_EINVAL;
    if (cfg.variant < 0 || cfg.variant > VARIANT_BLOCK)
        return BPIDA_EINVAL;
    if (cfg.variant >= tp::PSIMPLE && cfg.variant <= tp::BPSTATIC &&
        (cfg.width == 5 || cfg.count_all != 1 || cfg.budget != 0))
        return BPIDA_EINVAL;
    if (cfg.variant == VARIANT_BLOCK && cfg.width == 5)
        return BPIDA_EINVAL;
    if (cfg.count_all != 0 && cfg.count_all != 1)
        return BPIDA_EINVAL;
    return BPIDA_OK;
}

bpida_status dispatch(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                      uint64_t *out_nodes_per_iter, int *out_num_iters, int *out_status, uint64_t *out_solutions,
                      cudaStream_t st)
{
    switch (cfg.width) {
    case 3:
        return run_w<3>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status,
                        out_solutions, st);
    case 4:
        return run_w<4>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status,
                        out_solutions, st);
    default:
        return run_w<5>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status,
                        out_solutions, st);
    }
}

}  // namespace

extern "C" {

bpida_status bpida_solve_ex(const bpida_config *cfg_in, const uint64_t *boards, int n, int *out_len,
                            uint8_t *out_moves, uint64_t *out_nodes_per_iter, int *out_num_iters,
                            int *out_status, uint64_t *out_solutions, void *stream)
{
    Settings cfg;
    const bpida_status bad = parse_settings(cfg_in, n, cfg);
    if (bad != BPIDA_OK)
        return bad;
    if (n == 0)
        return BPIDA_OK;
    if (!boards || !out_len || !out_moves || !out_nodes_per_iter)
        return BPIDA_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t st = (cudaStream_t)stream;
    if (cfg.variant >= tp::PSIMPLE && cfg.variant <= tp::BPSTATIC) {
        tp::Settings ts;
        ts.width = cfg.width;
        ts.variant = cfg.variant;
        ts.threads = cfg.split_target;
        bpida_stats stats;
        std::memset(&stats, 0, sizeof stats);
        const bpida_status r = tp::solve(ts, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters,
                                         out_status, out_solutions, st, &stats);
        g_stats = stats;
        return r;
    }
    return dispatch(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status,
                    out_solutions, st);
}

bpida_status bpida_solve_pdb(const bpida_config *cfg_in, const bpida_pdb *pdb, const uint64_t *boards, int n,
                             int *out_len, uint8_t *out_moves, uint64_t *out_nodes_per_iter, int *out_num_iters,
                             int *out_status, uint64_t *out_solutions, void *stream)
{
    if (!pdb)
        return BPIDA_EINVAL;
    bpida_config c;
    std::memset(&c, 0, sizeof c);
    if (cfg_in)
        c = *cfg_in;
    else
        c.count_all = 1;
    if (c.width == 0)
        c.width = pdb->width;
    if (c.stack_entries != 0 && c.stack_entries != 256 && c.stack_entries != 384 && c.stack_entries != 512)
        return BPIDA_EINVAL;
    // 24-byte stack entries: 384 of them per warp keep six 4-warp blocks per SM
    if (c.stack_entries == 0)
        c.stack_entries = 384;
    Settings cfg;
    const bpida_status bad = parse_settings(&c, n, cfg);
    if (bad != BPIDA_OK)
        return bad;
    if (cfg.variant != 0 || cfg.width != pdb->width)
        return BPIDA_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return BPIDA_ECUDA;
    if (dev != pdb->dev)
        return BPIDA_EINVAL;
    cfg.pdb = pdb;
    if (n == 0)
        return BPIDA_OK;
    if (!boards || !out_len || !out_moves || !out_nodes_per_iter)
        return BPIDA_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    return dispatch(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status,
                    out_solutions, (cudaStream_t)stream);
}

bpida_status bpida_solve(const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                         uint64_t *out_nodes_per_iter, void *stream)
{
    return bpida_solve_ex(nullptr, boards, n, out_len, out_moves, out_nodes_per_iter, nullptr, nullptr, nullptr,
                          stream);
}

void bpida_set_timing(int on) { g_timing = on ? 1 : 0; }

int bpida_get_launch_log(double *ms, uint64_t *nodes, int cap)
{
    const int k = (int)g_launch_log.size();
    for (int i = 0; i < k && i < cap; ++i) {
        if (ms)
            ms[i] = g_launch_log[i].ms;
        if (nodes)
            nodes[i] = g_launch_log[i].nodes;
    }
    return k;
}

void bpida_set_fuse_nodes(uint64_t nodes) { g_fuse_nodes.store(nodes); }

void bpida_get_stats(bpida_stats *out)
{
    if (!out)
        return;
    bpida_stats s = g_stats;
    if (g_last.ws) {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_last.ws->last_call == g_last.call && g_last.ws->h_ctrl)
            fill_loop_stats(s, *g_last.ws->h_ctrl, true);
    }
    *out = s;
}

void bpida_release_workspace(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return;
    if (dev < (int)g_ws.size())
        for (Workspace *w : g_ws[dev])
            w->release();
    g_last.ws = nullptr;
    tp::release(dev);
    noalloc_forget(dev);
}

const char *bpida_status_str(int s)
{
    switch (s) {
    case BPIDA_OK: return "ok";
    case BPIDA_EINVAL: return "invalid argument or unsolvable board";
    case BPIDA_ENOMEM: return "device memory or queue capacity exceeded";
    case BPIDA_ESTACK: return "search stack bound exceeded";
    case BPIDA_EBUDGET: return "node budget exhausted";
    case BPIDA_ETIMEOUT: return "device wait timed out";
    case BPIDA_ECUDA: return "CUDA runtime error";
    case BPIDA_ELIMIT: return "solution length cap exceeded";
    case BPIDA_EINTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

}  // extern "C"
