// bpida_solve_noalloc: the 15-puzzle solve for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc (or any allocating routine) at the
// moment they want a solve: hosts whose device memory is entirely reserved
// up front by a framework's pool allocator, and latency-critical loops that
// cannot afford cudaMalloc's implicit device synchronisation. This entry
// point serves them: it runs the same kernels as bpida_solve_ex, driven from
// the host, with its whole workspace taken from one file-scope __device__
// array of BPIDA_NOALLOC_SCRATCH_BYTES. It never calls cudaMalloc, cudaFree,
// cudaMallocHost, a graph instantiation or an event creation. The caller
// still passes device buffers for the boards and all outputs.
//
// The array belongs to every GPU that loads this library, for the life of
// the process. Its device address is taken once per device, on the first
// call made with that device current (cudaGetSymbolAddress); a
// cudaDeviceReset makes that address stale, and bpida_release_workspace()
// forgets it so that the next call takes it again. Every call shares the
// array and leaves its contents behind; each call re-initialises everything
// it reads (control block, instance state, counters) before use. Calls that
// overlap on the GPU would race on the array; calls through this entry point
// are serialised by a lock and each one synchronises its stream before it
// returns.
#include "bpida.h"
#include "bpida_device.cuh"

#include <cstdio>
#include <cstring>
#include <mutex>

using namespace bp;

namespace {

typedef Rec<4> Rec4;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int NA_N = BPIDA_NOALLOC_MAX_BOARDS;  // boards per call
constexpr int NA_TCAP = 64;                     // frontier records per board and step
constexpr int NA_C = 4 * NA_TCAP + 4;           // splitter level capacity
constexpr int NA_WPB = 2;                       // warps per search block, one block per SM
constexpr int NA_S = 512;                       // shared-memory stack entries per warp
constexpr int NA_Q = 1 << 18;                   // records per hand-back queue

constexpr size_t OFF_CTRL = 0;
constexpr size_t OFF_DESC = OFF_CTRL + align256(sizeof(Ctrl));
constexpr size_t OFF_STATE = OFF_DESC + align256(sizeof(CallDesc));
constexpr size_t OFF_ACT0 = OFF_STATE + align256(sizeof(InstState<4>) * NA_N);
constexpr size_t OFF_ACT1 = OFF_ACT0 + align256(sizeof(unsigned) * NA_N);
constexpr size_t CTR_BYTES = (size_t)NA_N * (4 * sizeof(unsigned long long) + sizeof(int) + 2 * sizeof(unsigned));
constexpr size_t OFF_CTR = OFF_ACT1 + align256(sizeof(unsigned) * NA_N);
constexpr size_t OFF_COUNT = OFF_CTR + align256(CTR_BYTES);
constexpr size_t OFF_OFFSET = OFF_COUNT + align256(sizeof(int) * NA_N);
constexpr size_t OFF_SCRATCH = OFF_OFFSET + align256(sizeof(int) * NA_N);
constexpr size_t OFF_Q0 = OFF_SCRATCH + align256(sizeof(Rec4) * (size_t)NA_N * 2 * NA_C);
constexpr size_t OFF_Q1 = OFF_Q0 + align256(sizeof(Rec4) * (size_t)NA_Q);
constexpr size_t NA_BYTES = OFF_Q1 + align256(sizeof(Rec4) * (size_t)NA_Q);
static_assert(NA_BYTES <= (size_t)BPIDA_NOALLOC_SCRATCH_BYTES, "no-alloc workspace exceeds its array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[BPIDA_NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
unsigned char *g_na_base[NA_MAX_DEVICES] = {};

#define NA_CK(x)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            std::fprintf(stderr, "bpida_solve_noalloc: %s failed: %s\n", #x, cudaGetErrorString(e_)); \
            return BPIDA_ECUDA;                                                                   \
        }                                                                                         \
    } while (0)

}  // namespace

namespace bp {
// Forgets the array's device address on device dev (bpida_release_workspace).
void noalloc_forget(int dev)
{
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (dev >= 0 && dev < NA_MAX_DEVICES)
        g_na_base[dev] = nullptr;
}
}  // namespace bp

extern "C" bpida_status bpida_solve_noalloc(const uint64_t *boards, int n, int *out_len, uint8_t *out_moves,
                                            uint64_t *out_nodes_per_iter, int *out_num_iters,
                                            int *out_status, void *stream)
{
    if (n < 0 || n > NA_N) {
        std::fprintf(stderr, "bpida_solve_noalloc: n = %d is outside 0..%d\n", n, NA_N);
        return BPIDA_EINVAL;
    }
    if (n == 0)
        return BPIDA_OK;
    if (!boards || !out_len || !out_moves || !out_nodes_per_iter)
        return BPIDA_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        return BPIDA_EINVAL;
    if (!g_na_base[dev]) {
        // one-time set-up on this device: the host-side name of the array is
        // not a device address; ask the runtime for it
        unsigned char *p = nullptr;
        NA_CK(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch));
        g_na_base[dev] = p;
    }
    unsigned char *base = g_na_base[dev];
    int sms = 0;
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    Dev<4> d;
    std::memset(&d, 0, sizeof d);
    d.ctrl = (Ctrl *)(base + OFF_CTRL);
    d.desc = (const CallDesc *)(base + OFF_DESC);
    d.state = (InstState<4> *)(base + OFF_STATE);
    d.act0 = (unsigned *)(base + OFF_ACT0);
    d.act1 = (unsigned *)(base + OFF_ACT1);
    d.scratch = (Rec4 *)(base + OFF_SCRATCH);
    d.q0 = (Rec4 *)(base + OFF_Q0);
    d.q1 = (Rec4 *)(base + OFF_Q1);
    d.count = (int *)(base + OFF_COUNT);
    d.offset = (int *)(base + OFF_OFFSET);
    d.C = NA_C;
    d.Q = NA_Q;
    {
        unsigned char *p = base + OFF_CTR;
        d.cnt.search_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * NA_N;
        d.cnt.split_nodes = (unsigned long long *)p;
        p += sizeof(unsigned long long) * NA_N;
        d.cnt.goals = (unsigned long long *)p;
        p += sizeof(unsigned long long) * NA_N;
        d.cnt.budget_left = (unsigned long long *)p;
        p += sizeof(unsigned long long) * NA_N;
        d.cnt.fnext_off = (int *)p;
        p += sizeof(int) * NA_N;
        d.cnt.goal_origin = (unsigned *)p;
        p += sizeof(unsigned) * NA_N;
        d.cnt.aborted = (unsigned *)p;
    }
    const int grid = sms;
    const int threads = NA_WPB * 32;
    const size_t smem = SearchSmem<4>::TABLES + (size_t)NA_WPB * NA_S * WarpStack<4>::ENTRY_BYTES;
    d.tune.min_rounds = 64;
    d.tune.exit_threshold = (grid * NA_WPB) / 10 > 0 ? (grid * NA_WPB) / 10 : 1;
    d.tune.nodes_per_record = 4096;
    d.tune.target_cap = NA_TCAP;
    d.tune.target_path = NA_TCAP;
    d.tune.growth = 8;
    d.tune.min_pass_ns = 10000;
    d.lut = make_move_lut<4>();
    d.graph = 0;

    CallDesc desc;
    std::memset(&desc, 0, sizeof desc);
    desc.boards = boards;
    desc.out_len = out_len;
    desc.out_moves = out_moves;
    desc.out_nodes = (unsigned long long *)out_nodes_per_iter;
    desc.out_iters = out_num_iters;
    desc.out_status = out_status;
    desc.n = n;

    const dim3 b128(128), bsplit(SPLIT_THREADS), g_inst((n + 127) / 128);
    Ctrl h;
    k_set_desc<<<1, 1, 0, st>>>(desc, (CallDesc *)(base + OFF_DESC), d.ctrl);
    k_init<4><<<g_inst, b128, 0, st>>>(d);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&h, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    int n_active = h.n_active;
    while (n_active > 0) {
        k_split<4><<<n_active, bsplit, 0, st>>>(d);
        NA_CK(cudaGetLastError());
        for (;;) {
            k_search<4, NA_S><<<grid, threads, smem, st>>>(d);
            NA_CK(cudaGetLastError());
            NA_CK(cudaMemcpyAsync(&h, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            NA_CK(cudaStreamSynchronize(st));
            if (!h.pass_again)
                break;
        }
        k_advance<4><<<(n_active + 127) / 128, b128, 0, st>>>(d);
        NA_CK(cudaGetLastError());
        NA_CK(cudaMemcpyAsync(&h, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        n_active = h.step_again ? h.n_active : 0;
    }
    k_finalize<4><<<g_inst, b128, 0, st>>>(d);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&h, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (h.err & ERR_QUEUE)
        return BPIDA_ENOMEM;
    if (h.err)
        return BPIDA_EINTERNAL;
    return BPIDA_OK;
}
