// Host side of the GB300 Block-Parallel IDA* solver: the C ABI declared in
// include/bpida.h and the threshold loop of Algorithm 1 (BPIDA*).
//
// One solve call runs all of its instances together. Every step closes one
// f-limited iteration of every still-active instance (each at its own
// limit): k_split builds each instance's root set, k_scan/k_compact gather
// the root sets into one queue, k_search passes consume the queue with
// persistent warps (further passes only when warps handed work back), and
// k_advance records the iteration's node count and raises each limit to the
// smallest pruned f (or, once a goal was popped, walks down the first
// goal-bearing root to recover the solution path).
#include "bpida.h"
#include "bpida_device.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

using namespace bp;

namespace {

thread_local bpida_stats g_stats;
thread_local int g_timing = 0;
std::mutex g_mu;

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
};

cudaError_t ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
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

struct Workspace {
    DevBuf state, act0, act1, ctr, scratch, count, offset, q0, q1, ctrl;
    Ctrl *h_ctrl = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void release()
    {
        DevBuf *all[] = {&state, &act0, &act1, &ctr, &scratch, &count, &offset, &q0, &q1, &ctrl};
        for (DevBuf *b : all) {
            if (b->p)
                cudaFree(b->p);
            b->p = nullptr;
            b->n = 0;
        }
        if (h_ctrl)
            cudaFreeHost(h_ctrl);
        h_ctrl = nullptr;
        if (ev0)
            cudaEventDestroy(ev0);
        if (ev1)
            cudaEventDestroy(ev1);
        ev0 = ev1 = nullptr;
    }
};

std::vector<Workspace *> g_ws;

Workspace *workspace_for(int dev)
{
    if ((int)g_ws.size() <= dev)
        g_ws.resize(dev + 1, nullptr);
    if (!g_ws[dev])
        g_ws[dev] = new Workspace();
    return g_ws[dev];
}

// Manhattan move table (see MoveLut): for blank position p and move m,
// bit 0 = legal, bit t = tile t moves away from its goal cell.
template <int W> MoveLut<W> make_lut()
{
    MoveLut<W> L;
    std::memset(&L, 0, sizeof L);
    const int N = W * W;
    const int dr[4] = {-1, 0, 0, 1}, dc[4] = {0, -1, 1, 0};
    for (int p = 0; p < N; ++p) {
        const int r = p / W, c = p % W;
        for (int m = 0; m < 4; ++m) {
            const int rr = r + dr[m], cc = c + dc[m];
            if (rr < 0 || rr >= W || cc < 0 || cc >= W)
                continue;
            uint32_t e = 1u;
            for (int t = 1; t < N; ++t) {
                const int gr = t / W, gc = t % W;
                const int before = std::abs(rr - gr) + std::abs(cc - gc);
                const int after = std::abs(r - gr) + std::abs(c - gc);
                if (after > before)
                    e |= 1u << t;
            }
            L.e[p][m] = e;
        }
    }
    return L;
}

struct Settings {
    int width, count_all, split_target, wpb, S, exit_pct, min_rounds;
    uint64_t budget;
};

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            std::fprintf(stderr, "bpida: %s failed: %s\n", #x, cudaGetErrorString(e_));          \
            return e_ == cudaErrorMemoryAllocation ? BPIDA_ENOMEM : BPIDA_ECUDA;                  \
        }                                                                                         \
    } while (0)

template <int W, int S>
bpida_status run(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                 uint64_t *out_nodes, int *out_iters, int *out_status, cudaStream_t st)
{
    typedef typename Geo<W>::B B;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    Workspace &ws = *workspace_for(dev);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    const int wpb = cfg.wpb;
    const int threads = wpb * 32;
    const size_t smem = SharedLut<W>::BYTES + (size_t)wpb * S * WarpStack<W>::ENTRY_BYTES;
    CK(cudaFuncSetAttribute(k_search<W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int bpsm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_search<W, S>, threads, smem));
    if (bpsm < 1)
        return BPIDA_EINVAL;
    const int grid = sms * bpsm;
    const int total_warps = grid * wpb;

    int tcap = cfg.split_target;
    if (tcap <= 0)
        tcap = std::max(2, std::min(16384, (1 << 21) / std::max(n, 1)));
    const int C = 4 * tcap + 4;
    const size_t nrec_region = (size_t)n * 2 * C;
    // hand-back queue: every warp's stack plus its unfinished chunk, with
    // room for overflow spills (each spill moves S/2 entries); overflowing it
    // is detected and reported as BPIDA_ENOMEM
    const size_t Q = std::max({(size_t)n * C, (size_t)total_warps * (S + 32) * 4, (size_t)1 << 24}) + 1024;
    if (Q > (size_t)INT_MAX / 2)
        return BPIDA_ENOMEM;

    CK(ensure(ws.state, sizeof(InstState<W>) * n));
    CK(ensure(ws.act0, sizeof(unsigned) * n));
    CK(ensure(ws.act1, sizeof(unsigned) * n));
    const size_t ctr_bytes = (size_t)n * (3 * sizeof(unsigned long long) + sizeof(int) + sizeof(unsigned));
    CK(ensure(ws.ctr, ctr_bytes));
    CK(ensure(ws.scratch, sizeof(Rec<W>) * nrec_region));
    CK(ensure(ws.count, sizeof(int) * n));
    CK(ensure(ws.offset, sizeof(int) * n));
    CK(ensure(ws.q0, sizeof(Rec<W>) * Q));
    CK(ensure(ws.q1, sizeof(Rec<W>) * Q));
    CK(ensure(ws.ctrl, sizeof(Ctrl)));
    if (!ws.h_ctrl)
        CK(cudaMallocHost((void **)&ws.h_ctrl, sizeof(Ctrl)));
    if (!ws.ev0) {
        CK(cudaEventCreate(&ws.ev0));
        CK(cudaEventCreate(&ws.ev1));
    }

    Counters cnt;
    {
        char *p = (char *)ws.ctr.p;
        cnt.search_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        cnt.split_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        cnt.goals = (unsigned long long *)p;
        p += sizeof(unsigned long long) * n;
        cnt.fnext_off = (int *)p;
        p += sizeof(int) * n;
        cnt.goal_origin = (unsigned *)p;
    }
    Tune tune;
    tune.min_rounds = cfg.min_rounds;
    tune.exit_threshold = std::max(1, (int)((long long)total_warps * cfg.exit_pct / 100));
    tune.nodes_per_record = 4096;
    tune.target_cap = tcap;
    tune.target_path = std::min(tcap, 4096);
    tune.growth = 8;

    const MoveLut<W> lut = make_lut<W>();
    Ctrl *ctrl = (Ctrl *)ws.ctrl.p;
    InstState<W> *state = (InstState<W> *)ws.state.p;
    unsigned *act[2] = {(unsigned *)ws.act0.p, (unsigned *)ws.act1.p};
    Rec<W> *scratch = (Rec<W> *)ws.scratch.p;
    Rec<W> *q[2] = {(Rec<W> *)ws.q0.p, (Rec<W> *)ws.q1.p};
    int *count = (int *)ws.count.p, *offset = (int *)ws.offset.p;

    bpida_stats stats;
    std::memset(&stats, 0, sizeof stats);
    stats.grid_blocks = grid;
    stats.block_threads = threads;
    stats.sm_count = sms;

    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    {
        InitArgs<W> ia{boards, n, state, act[0], ctrl, out_moves, (unsigned long long *)out_nodes};
        k_init<W><<<(n + 127) / 128, 128, 0, st>>>(ia);
        CK(cudaGetLastError());
        stats.launches++;
    }
    CK(cudaMemcpyAsync(ws.h_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int n_active = ws.h_ctrl->n_active;
    int cur = 0;
    bpida_status abort_status = BPIDA_OK;

    while (n_active > 0) {
        SplitArgs<W> sa{act[cur], state, scratch, C, count, cnt, lut};
        k_split<W><<<n_active, 256, 0, st>>>(sa);
        CK(cudaGetLastError());
        k_scan<<<1, 1024, 0, st>>>(count, offset, ctrl);
        CK(cudaGetLastError());
        k_compact<W><<<n_active, 128, 0, st>>>(scratch, C, count, offset, q[0]);
        CK(cudaGetLastError());
        stats.launches += 3;
        int qi = 0;
        for (;;) {
            SearchArgs<W> a{q[qi], q[qi ^ 1], (int)Q, ctrl, cnt, tune, lut};
            if (g_timing)
                CK(cudaEventRecord(ws.ev0, st));
            k_search<W, S><<<grid, threads, smem, st>>>(a);
            CK(cudaGetLastError());
            if (g_timing)
                CK(cudaEventRecord(ws.ev1, st));
            stats.passes++;
            stats.launches++;
            CK(cudaMemcpyAsync(ws.h_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (g_timing) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1));
                stats.search_ms += ms;
            }
            if (ws.h_ctrl->err & ERR_QUEUE) {
                abort_status = BPIDA_ENOMEM;
                break;
            }
            if (ws.h_ctrl->out_count == 0)
                break;
            k_next_pass<<<1, 1, 0, st>>>(ctrl);
            CK(cudaGetLastError());
            stats.launches++;
            qi ^= 1;
        }
        if (abort_status != BPIDA_OK)
            break;
        AdvanceArgs<W> aa{act[cur], act[cur ^ 1], state, scratch, C, count, offset, cnt, ctrl, tune,
                          (unsigned long long)cfg.budget, out_moves, (unsigned long long *)out_nodes};
        k_advance<W><<<(n_active + 127) / 128, 128, 0, st>>>(aa);
        CK(cudaGetLastError());
        k_step_end<<<1, 1, 0, st>>>(ctrl);
        CK(cudaGetLastError());
        stats.launches += 2;
        CK(cudaMemcpyAsync(ws.h_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats.steps++;
        n_active = ws.h_ctrl->n_active;
        cur ^= 1;
    }
    k_finalize<W><<<(n + 127) / 128, 128, 0, st>>>(state, n, out_len, out_iters, out_status,
                                                   (int)abort_status);
    CK(cudaGetLastError());
    stats.launches++;
    CK(cudaMemcpyAsync(ws.h_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stats.records = ws.h_ctrl->records_total;
    stats.handed_back = ws.h_ctrl->handed_back_total;
    stats.search_nodes = ws.h_ctrl->search_nodes_total;
    stats.spills = ws.h_ctrl->spills;
    stats.max_handed_back = ws.h_ctrl->max_out;
    g_stats = stats;
    if (abort_status != BPIDA_OK)
        return abort_status;
    if (ws.h_ctrl->err & ERR_INTERNAL)
        return BPIDA_EINTERNAL;
    return BPIDA_OK;
}

template <int W>
bpida_status run_w(const Settings &cfg, const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                   uint64_t *out_nodes, int *out_iters, int *out_status, cudaStream_t st)
{
    switch (cfg.S) {
    case 256: return run<W, 256>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, st);
    case 1024: return run<W, 1024>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, st);
    default: return run<W, 512>(cfg, boards, n, out_len, out_moves, out_nodes, out_iters, out_status, st);
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

bpida_status bpida_solve_ex(const bpida_config *cfg_in, const uint64_t *boards, int n, int *out_len,
                            uint8_t *out_moves, uint64_t *out_nodes_per_iter, int *out_num_iters,
                            int *out_status, void *stream)
{
    Settings cfg;
    cfg.width = (cfg_in && cfg_in->width) ? cfg_in->width : 4;
    cfg.count_all = cfg_in ? cfg_in->count_all : 1;
    cfg.split_target = cfg_in ? cfg_in->split_target : 0;
    cfg.wpb = (cfg_in && cfg_in->warps_per_block > 0) ? cfg_in->warps_per_block : 4;
    cfg.S = (cfg_in && cfg_in->stack_entries > 0) ? cfg_in->stack_entries : 512;
    cfg.exit_pct = (cfg_in && cfg_in->exit_fraction_pct > 0) ? cfg_in->exit_fraction_pct : 25;
    cfg.min_rounds = (cfg_in && cfg_in->min_rounds > 0) ? cfg_in->min_rounds : 64;
    cfg.budget = cfg_in ? cfg_in->node_budget : 0;
    if (cfg.width < 3 || cfg.width > 5 || n < 0)
        return BPIDA_EINVAL;
    if (cfg.S != 256 && cfg.S != 512 && cfg.S != 1024)
        return BPIDA_EINVAL;
    if (cfg.wpb < 1 || cfg.wpb > 32 || cfg.exit_pct > 100 || cfg.split_target < 0)
        return BPIDA_EINVAL;
    if (cfg.count_all != 1)
        return BPIDA_EINVAL;  // only the all-solutions mode is implemented
    if (n == 0)
        return BPIDA_OK;
    if (!boards || !out_len || !out_moves || !out_nodes_per_iter)
        return BPIDA_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t st = (cudaStream_t)stream;
    switch (cfg.width) {
    case 3: return run_w<3>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status, st);
    case 4: return run_w<4>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status, st);
    default: return run_w<5>(cfg, boards, n, out_len, out_moves, out_nodes_per_iter, out_num_iters, out_status, st);
    }
}

bpida_status bpida_solve(const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                         uint64_t *out_nodes_per_iter, void *stream)
{
    return bpida_solve_ex(nullptr, boards, n, out_len, out_moves, out_nodes_per_iter, nullptr, nullptr,
                          stream);
}

void bpida_set_timing(int on) { g_timing = on ? 1 : 0; }

void bpida_get_stats(bpida_stats *out)
{
    if (out)
        *out = g_stats;
}

void bpida_release_workspace(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return;
    if (dev < (int)g_ws.size() && g_ws[dev])
        g_ws[dev]->release();
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
