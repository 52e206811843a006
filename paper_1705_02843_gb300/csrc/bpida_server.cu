// Continuous-batching solve service (the "serving" form of the batched
// solver): requests arrive at any time, are admitted into free instance
// slots between threshold steps, and share every search pass with the
// requests already on the GPU; each request keeps its own f-limit and its
// search state stays in device memory across thresholds. Results are posted
// to a completion queue as soon as their instance finishes.
//
// One host thread per server drives the device loop:
//   admit (k_admit) -> one threshold step (k_split, k_search passes,
//   k_advance) -> harvest the instances that finished (k_pack)
// A step is time-sliced: once it has run for the slice, the search passes
// stop and the open nodes of every unfinished iteration are carried into the
// next step (k_carry_mark), so that requests whose iterations are short
// advance, finish and free their slots without waiting for the longest
// iteration of the batch, and new requests join sooner.
// using the same kernels as bpida_solve_ex. The number of slots is bounded
// by the frontier memory the caller grants (each slot owns 2*C frontier
// records), so admission is by frontier memory.
#include "bpida.h"
#include "bpida_device.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

using namespace bp;

namespace {

constexpr int SV_W = 4;
constexpr int SV_S = 384;
constexpr int SV_WPB = 4;
constexpr int SV_MAXLEN = Geo<SV_W>::MAXLEN;
constexpr int SV_MAXIT = Geo<SV_W>::MAXIT;

struct Packed {
    int len, iters, status, slot;
    unsigned long long solutions;
    uint8_t moves[SV_MAXLEN];
    unsigned long long nodes[SV_MAXIT];
};

// Gathers the results of the instances in the done list.
__global__ void k_pack(const Dev<SV_W> a, Packed *out)
{
    const CallDesc dsc = *a.desc;
    const int j = blockIdx.x;
    if (j >= a.ctrl->n_done)
        return;
    const unsigned i = a.done_list[j];
    const InstState<SV_W> st = a.state[i];
    Packed &o = out[j];
    for (int q = threadIdx.x; q < SV_MAXLEN; q += blockDim.x)
        o.moves[q] = dsc.out_moves[(size_t)i * SV_MAXLEN + q];
    for (int q = threadIdx.x; q < SV_MAXIT; q += blockDim.x)
        o.nodes[q] = dsc.out_nodes[(size_t)i * SV_MAXIT + q];
    if (threadIdx.x == 0) {
        const bool solved = st.mode == MODE_DONE && st.status == 0;
        o.len = solved ? st.length : -1;
        o.iters = st.rows;
        o.status = st.mode == MODE_DONE ? st.status : 8;
        o.slot = (int)i;
        o.solutions = solved ? st.solutions : 0ull;
    }
}

double now_s()
{
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id;
    uint64_t board;
    double submit;
};

}  // namespace

struct bpida_server {
    int dev = 0;
    int max_slots = 0;
    int grid = 0, threads = 0;
    size_t smem = 0;
    cudaStream_t st = nullptr;
    void *mem = nullptr;
    Dev<SV_W> d;
    unsigned *d_admit_slot = nullptr;
    uint64_t *d_admit_board = nullptr;
    Packed *d_packed = nullptr;
    unsigned *h_admit_slot = nullptr;
    uint64_t *h_admit_board = nullptr;
    Packed *h_packed = nullptr;
    Ctrl *h_ctrl = nullptr;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::deque<bpida_result> done;
    std::vector<int> free_slots;
    std::vector<Req> in_slot;
    int in_flight = 0;
    bool stop = false;
    std::atomic<bool> failed{false};
    std::atomic<long long> slice_ns{2000000};
    bpida_server_stats stats;
    std::thread th;

    bool step_error(const char *what, cudaError_t e)
    {
        std::fprintf(stderr, "bpida server: %s: %s\n", what, cudaGetErrorString(e));
        failed = true;
        return false;
    }
    void loop();
    bool device_step(int admitted);
};

#define SV_CK(x)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess)                                                                    \
            return step_error(#x, e_);                                                            \
    } while (0)

// One round of the device loop: admit `admitted` staged requests, run one
// threshold step for every active instance, harvest what finished.
bool bpida_server::device_step(int admitted)
{
    if (admitted > 0) {
        SV_CK(cudaMemcpyAsync(d_admit_slot, h_admit_slot, sizeof(unsigned) * admitted, cudaMemcpyHostToDevice, st));
        SV_CK(cudaMemcpyAsync(d_admit_board, h_admit_board, sizeof(uint64_t) * admitted, cudaMemcpyHostToDevice, st));
        k_admit<SV_W><<<(admitted + 127) / 128, 128, 0, st>>>(d, d_admit_slot, d_admit_board, admitted);
        SV_CK(cudaGetLastError());
    }
    SV_CK(cudaMemcpyAsync(h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SV_CK(cudaStreamSynchronize(st));
    const int n_active = h_ctrl->n_active;
    uint64_t passes = 0, steps = 0, sliced = 0;
    d.tune.step_ns = (unsigned long long)std::max(0ll, slice_ns.load());
    if (n_active > 0) {
        k_split<SV_W><<<n_active, SPLIT_THREADS, 0, st>>>(d);
        SV_CK(cudaGetLastError());
        for (;;) {
            k_search<SV_W, SV_S><<<grid, threads, smem, st>>>(d);
            SV_CK(cudaGetLastError());
            SV_CK(cudaMemcpyAsync(h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            SV_CK(cudaStreamSynchronize(st));
            ++passes;
            if (!h_ctrl->pass_again)
                break;
        }
        if (h_ctrl->n_carry > 0) {
            k_carry_mark<SV_W><<<(h_ctrl->n_carry + 255) / 256, 256, 0, st>>>(d);
            SV_CK(cudaGetLastError());
            ++sliced;
        }
        k_advance<SV_W><<<(n_active + 127) / 128, 128, 0, st>>>(d);
        SV_CK(cudaGetLastError());
        // the step guard of the solve loop counts steps per call; a server
        // runs without end, so it restarts the count every step
        SV_CK(cudaMemsetAsync(&d.ctrl->steps, 0, sizeof(int), st));
        ++steps;
    }
    SV_CK(cudaMemcpyAsync(h_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SV_CK(cudaStreamSynchronize(st));
    if (h_ctrl->err) {
        std::fprintf(stderr, "bpida server: device error bits %d\n", h_ctrl->err);
        failed = true;
        return false;
    }
    const int n_done = h_ctrl->n_done;
    {
        std::lock_guard<std::mutex> lock(mu);
        stats.passes += passes;
        stats.steps += steps;
        stats.sliced_steps += sliced;
        stats.max_active = std::max(stats.max_active, n_active);
    }
    if (n_done > 0) {
        k_pack<<<n_done, 64, 0, st>>>(d, d_packed);
        SV_CK(cudaGetLastError());
        SV_CK(cudaMemcpyAsync(h_packed, d_packed, sizeof(Packed) * n_done, cudaMemcpyDeviceToHost, st));
        SV_CK(cudaMemsetAsync(&d.ctrl->n_done, 0, sizeof(int), st));
        SV_CK(cudaStreamSynchronize(st));
        const double t = now_s();
        std::lock_guard<std::mutex> lock(mu);
        for (int j = 0; j < n_done; ++j) {
            const Packed &pk = h_packed[j];
            const Req &rq = in_slot[pk.slot];
            bpida_result r;
            std::memset(&r, 0, sizeof r);
            r.req_id = rq.id;
            r.status = pk.status;
            r.length = pk.len;
            r.num_iters = pk.iters;
            r.submit_time_s = rq.submit;
            r.done_time_s = t;
            std::memcpy(r.moves, pk.moves, sizeof r.moves);
            for (int q = 0; q < SV_MAXIT; ++q)
                r.nodes_per_iter[q] = pk.nodes[q];
            r.solutions = pk.solutions;
            done.push_back(r);
            free_slots.push_back(pk.slot);
            --in_flight;
            stats.completed++;
        }
    }
    return true;
}

void bpida_server::loop()
{
    cudaSetDevice(dev);
    for (;;) {
        int admitted = 0;
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stop)
                break;
            while (!pending.empty() && !free_slots.empty()) {
                const Req rq = pending.front();
                pending.pop_front();
                const int slot = free_slots.back();
                free_slots.pop_back();
                in_slot[slot] = rq;
                h_admit_slot[admitted] = (unsigned)slot;
                h_admit_board[admitted] = rq.board;
                ++admitted;
            }
            stats.admitted += admitted;
            const bool idle = admitted == 0 && in_flight == (int)pending.size();
            if (idle) {
                // nothing on the device: wait for a request (or stop)
                cv.wait_for(lock, std::chrono::milliseconds(2), [&] { return stop || !pending.empty(); });
                continue;
            }
        }
        if (!device_step(admitted)) {
            // fail everything in flight, then keep refusing work
            std::lock_guard<std::mutex> lock(mu);
            const double t = now_s();
            for (int s = 0; s < max_slots; ++s) {
                bool is_free = std::find(free_slots.begin(), free_slots.end(), s) != free_slots.end();
                if (is_free)
                    continue;
                bpida_result r;
                std::memset(&r, 0, sizeof r);
                r.req_id = in_slot[s].id;
                r.status = BPIDA_ECUDA;
                r.length = -1;
                r.submit_time_s = in_slot[s].submit;
                r.done_time_s = t;
                done.push_back(r);
                free_slots.push_back(s);
            }
            in_flight = (int)pending.size();
            break;
        }
    }
}

extern "C" {

bpida_server *bpida_server_create(const bpida_config *cfg, size_t frontier_bytes, int max_slots)
{
    if ((cfg && cfg->width && cfg->width != 4) || max_slots <= 0)
        return nullptr;
    const int tcap = (cfg && cfg->split_target > 0) ? cfg->split_target : 256;
    const int C = 4 * tcap + 4;
    const size_t per_slot = sizeof(Rec<SV_W>) * 2 * (size_t)C;
    const int slots = (int)std::min<size_t>((size_t)max_slots, frontier_bytes / per_slot);
    if (slots < 1)
        return nullptr;
    bpida_server *sv = new bpida_server();
    std::memset(&sv->stats, 0, sizeof sv->stats);
    cudaGetDevice(&sv->dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->dev);
    sv->max_slots = slots;
    sv->threads = SV_WPB * 32;
    sv->smem = SearchSmem<SV_W>::TABLES + (size_t)SV_WPB * SV_S * WarpStack<SV_W>::ENTRY_BYTES;
    int bpsm = 0, smem_max = 0;
    // the device maximum, as the solve path sets it: the kernel is shared
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, sv->dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_search<SV_W, SV_S>) == cudaSuccess)
        smem_max -= (int)fa.sharedSizeBytes;  // less the kernel's static shared memory
    if (cudaFuncSetAttribute(k_search<SV_W, SV_S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_search<SV_W, SV_S>, sv->threads, sv->smem) !=
            cudaSuccess ||
        bpsm < 1) {
        delete sv;
        return nullptr;
    }
    sv->grid = sms * bpsm;
    const int total_warps = sv->grid * SV_WPB;
    const int ovf_cap = 0;  // 15-puzzle: no overflow stacks
    const size_t Q = std::max({(size_t)slots * C, (size_t)total_warps * (SV_S + ovf_cap + 32) * 2, (size_t)1 << 24}) + 1024;

    // one allocation carved into the workspace
    const size_t n = (size_t)slots;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_ctrl = take(sizeof(Ctrl)), o_desc = take(sizeof(CallDesc));
    const size_t o_state = take(sizeof(InstState<SV_W>) * n), o_act0 = take(4 * n), o_act1 = take(4 * n);
    const size_t o_ctr = take(n * (4 * 8 + 4 + 4 + 4)), o_count = take(4 * n), o_offset = take(4 * n);
    const size_t o_scr = take(sizeof(Rec<SV_W>) * n * 2 * C), o_q0 = take(sizeof(Rec<SV_W>) * Q),
                 o_q1 = take(sizeof(Rec<SV_W>) * Q);
    const size_t o_done = take(4 * n), o_aslot = take(4 * n), o_aboard = take(8 * n), o_packed = take(sizeof(Packed) * n);
    const size_t o_len = take(4 * n), o_moves = take(SV_MAXLEN * n), o_nodes = take(8 * SV_MAXIT * n),
                 o_iters = take(4 * n), o_status = take(4 * n);
    const size_t o_ovf = take((size_t)total_warps * ovf_cap * WarpStack<SV_W>::ENTRY_BYTES);
    const size_t o_carry = take(4 * n), o_fbase = take(4 * n), o_fcount = take(4 * n);
    if (cudaMalloc(&sv->mem, off) != cudaSuccess) {
        delete sv;
        return nullptr;
    }
    char *b = (char *)sv->mem;
    Dev<SV_W> &d = sv->d;
    std::memset(&d, 0, sizeof d);
    d.ctrl = (Ctrl *)(b + o_ctrl);
    d.desc = (const CallDesc *)(b + o_desc);
    d.state = (InstState<SV_W> *)(b + o_state);
    d.act0 = (unsigned *)(b + o_act0);
    d.act1 = (unsigned *)(b + o_act1);
    d.scratch = (Rec<SV_W> *)(b + o_scr);
    d.q0 = (Rec<SV_W> *)(b + o_q0);
    d.q1 = (Rec<SV_W> *)(b + o_q1);
    d.count = (int *)(b + o_count);
    d.offset = (int *)(b + o_offset);
    d.C = C;
    d.Q = (int)Q;
    d.ovf = (unsigned char *)(b + o_ovf);
    d.ovf_cap = ovf_cap;
    d.slice = 1;
    d.carry = (unsigned *)(b + o_carry);
    d.fbase = (int *)(b + o_fbase);
    d.fcount = (int *)(b + o_fcount);
    {
        char *p = b + o_ctr;
        d.cnt.search_nodes = (unsigned long long *)p;
        p += 8 * n;
        d.cnt.split_nodes = (unsigned long long *)p;
        p += 8 * n;
        d.cnt.goals = (unsigned long long *)p;
        p += 8 * n;
        d.cnt.budget_left = (unsigned long long *)p;
        p += 8 * n;
        d.cnt.fnext_off = (int *)p;
        p += 4 * n;
        d.cnt.goal_origin = (unsigned *)p;
        p += 4 * n;
        d.cnt.aborted = (unsigned *)p;
    }
    const int exit_pct = (cfg && cfg->exit_fraction_pct > 0) ? cfg->exit_fraction_pct : 10;
    d.tune.min_rounds = (cfg && cfg->min_rounds > 0) ? cfg->min_rounds : 64;
    d.tune.exit_threshold = std::max(1, total_warps * exit_pct / 100);
    d.tune.nodes_per_record = 4096;
    d.tune.target_cap = tcap;
    d.tune.target_path = std::min(tcap, 4096);
    d.tune.growth = 8;
    d.tune.min_pass_ns = 10000;
    d.lut = make_move_lut<SV_W>();
    d.graph = 0;
    d.done_list = (unsigned *)(b + o_done);
    sv->d_admit_slot = (unsigned *)(b + o_aslot);
    sv->d_admit_board = (uint64_t *)(b + o_aboard);
    sv->d_packed = (Packed *)(b + o_packed);

    CallDesc desc;
    std::memset(&desc, 0, sizeof desc);
    desc.out_len = (int *)(b + o_len);
    desc.out_moves = (uint8_t *)(b + o_moves);
    desc.out_nodes = (unsigned long long *)(b + o_nodes);
    desc.out_iters = (int *)(b + o_iters);
    desc.out_status = (int *)(b + o_status);
    desc.n = slots;

    bool ok = cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sv->h_admit_slot, 4 * n) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sv->h_admit_board, 8 * n) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sv->h_packed, sizeof(Packed) * n) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sv->h_ctrl, sizeof(Ctrl)) == cudaSuccess;
    ok = ok && cudaMemsetAsync(d.carry, 0, 4 * n, sv->st) == cudaSuccess;
    if (ok) {
        k_set_desc<<<1, 1, 0, sv->st>>>(desc, (CallDesc *)(b + o_desc), d.ctrl);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(sv->st) == cudaSuccess;
    }
    if (!ok) {
        bpida_server_destroy(sv);
        return nullptr;
    }
    sv->in_slot.resize(slots);
    sv->free_slots.reserve(slots);
    for (int s = slots - 1; s >= 0; --s)
        sv->free_slots.push_back(s);
    sv->stats.slots = slots;
    sv->th = std::thread([sv] { sv->loop(); });
    return sv;
}

bpida_status bpida_server_submit(bpida_server *sv, const uint64_t *host_board, uint64_t req_id)
{
    if (!sv || !host_board)
        return BPIDA_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->failed || sv->stop)
        return BPIDA_ECUDA;
    sv->pending.push_back(Req{req_id, *host_board, now_s()});
    sv->in_flight++;
    sv->stats.submitted++;
    sv->cv.notify_one();
    return BPIDA_OK;
}

int bpida_server_poll(bpida_server *sv, bpida_result *out, int max)
{
    if (!sv || !out || max <= 0)
        return 0;
    std::lock_guard<std::mutex> lock(sv->mu);
    int k = 0;
    while (k < max && !sv->done.empty()) {
        out[k++] = sv->done.front();
        sv->done.pop_front();
    }
    return k;
}

int bpida_server_in_flight(bpida_server *sv)
{
    if (!sv)
        return 0;
    std::lock_guard<std::mutex> lock(sv->mu);
    return sv->in_flight;
}

void bpida_server_get_stats(bpida_server *sv, bpida_server_stats *out)
{
    if (!sv || !out)
        return;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
}

double bpida_server_clock(void) { return now_s(); }

void bpida_server_set_time_slice(bpida_server *sv, int microseconds)
{
    if (sv)
        sv->slice_ns = microseconds > 0 ? 1000ll * microseconds : 0ll;
}

void bpida_server_destroy(bpida_server *sv)
{
    if (!sv)
        return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->th.joinable())
        sv->th.join();
    if (sv->st)
        cudaStreamSynchronize(sv->st);
    if (sv->mem)
        cudaFree(sv->mem);
    if (sv->h_admit_slot)
        cudaFreeHost(sv->h_admit_slot);
    if (sv->h_admit_board)
        cudaFreeHost(sv->h_admit_board);
    if (sv->h_packed)
        cudaFreeHost(sv->h_packed);
    if (sv->h_ctrl)
        cudaFreeHost(sv->h_ctrl);
    if (sv->st)
        cudaStreamDestroy(sv->st);
    delete sv;
}

}  // extern "C"
