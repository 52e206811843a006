/*
 * Oracle: plain sequential IDA* for the (W*W-1)-puzzle with the Manhattan
 * distance heuristic, W in {3, 4, 5}.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it. It shares no code with the CUDA path.
 *
 * What it computes (Horie & Fukunaga, "Block-Parallel IDA* for GPUs"):
 *   - the f-limited depth-first search of Algorithm 2 with dynamic load
 *     balancing switched off (the paper's sequential Solver C, Section 3):
 *     pop s; if s is a goal, report it; otherwise, for every applicable
 *     action, f_new = g(s) + cost(a) + h(t); push t if f_new <= limit,
 *     else f_next = min(f_next, f_new);
 *   - the iteration driver of Algorithms 1/2: the first limit is h(start)
 *     and every later limit is the smallest pruned f of the previous
 *     iteration, until an iteration reaches a goal;
 *   - the all-optimal-solutions mode of Section 6 (the final iteration is
 *     run to completion, so its node count does not depend on node order).
 *
 * Readings where the paper is silent (each listed with its reason in the
 * design notes): goal = blank at position 0 and tile t at position t;
 * blank moves tried in the order U, L, R, D; the inverse of the previous
 * move is never applied (parent pruning); a node is counted ("expanded")
 * when it is popped with f <= limit, the root and goal nodes included; a
 * goal is tested when popped and is not expanded further; cost(a) = 1.
 *
 * Parity status: pinned. The tests check this file against a brute-force
 * breadth-first search of all 181,440 reachable 8-puzzle states (optimal
 * lengths), Manhattan admissibility and consistency on every 8-puzzle edge,
 * hand-worked node counts, an independent memoised tree-size recurrence,
 * the +2 threshold invariant and replay of every returned move sequence.
 *
 * Boards are plain arrays: t[p] = tile at position p, 0 = blank. The
 * heuristic is recomputed from scratch (sum over tiles of |dr| + |dc|) at
 * every generated node.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>
#include <pthread.h>

#define OR_MAX_W 5
#define OR_MAX_N (OR_MAX_W * OR_MAX_W)
#define OR_MAX_PATH 512

/* status codes returned per instance */
#define OR_OK 0
#define OR_INVALID 1      /* not a permutation, or not in the goal's parity class */
#define OR_BUDGET 4       /* node budget exhausted before a solution */
#define OR_LIMIT 7        /* iteration or length cap reached before a solution */
#define OR_BADARG 8

typedef struct {
    int W, N;
    int row[OR_MAX_N], col[OR_MAX_N];
    uint8_t t[OR_MAX_N];
    int blank;
    int limit;
    int fnext;
    int count_all;
    int stop;
    int budget_hit;
    uint64_t nodes_it;
    uint64_t total;
    uint64_t budget;
    uint64_t solutions;
    int have_path;
    uint8_t path[OR_MAX_PATH];
    uint8_t first[OR_MAX_PATH];
} ctx_t;

/* Manhattan distance: sum over non-blank tiles of |row - goal row| +
 * |col - goal col|; tile v's goal position is v. */
static int manhattan(const ctx_t *c)
{
    int h = 0;
    for (int p = 0; p < c->N; ++p) {
        int v = c->t[p];
        if (v == 0)
            continue;
        int dr = c->row[p] - c->row[v];
        int dc = c->col[p] - c->col[v];
        h += (dr < 0 ? -dr : dr) + (dc < 0 ? -dc : dc);
    }
    return h;
}

static int is_goal(const ctx_t *c)
{
    for (int p = 0; p < c->N; ++p)
        if (c->t[p] != p)
            return 0;
    return 1;
}

/* New blank position after move m (U, L, R, D), or -1 if it leaves the board. */
static int blank_target(const ctx_t *c, int p, int m)
{
    int r = c->row[p], q = c->col[p];
    switch (m) {
    case 0: return r > 0 ? p - c->W : -1;
    case 1: return q > 0 ? p - 1 : -1;
    case 2: return q < c->W - 1 ? p + 1 : -1;
    case 3: return r < c->W - 1 ? p + c->W : -1;
    }
    return -1;
}

static void dfs(ctx_t *c, int g, int last)
{
    c->nodes_it++;
    c->total++;
    if (c->budget && c->total > c->budget) {
        c->budget_hit = 1;
        c->stop = 1;
        return;
    }
    if (is_goal(c)) {
        c->solutions++;
        if (!c->have_path) {
            memcpy(c->first, c->path, (size_t)g);
            c->have_path = 1;
        }
        if (!c->count_all)
            c->stop = 1;
        return;
    }
    for (int m = 0; m < 4; ++m) {
        if (last >= 0 && m == 3 - last)
            continue;
        int p = c->blank;
        int np = blank_target(c, p, m);
        if (np < 0)
            continue;
        /* the tile at np slides into the blank */
        c->t[p] = c->t[np];
        c->t[np] = 0;
        c->blank = np;
        int f = g + 1 + manhattan(c);
        if (f <= c->limit) {
            c->path[g] = (uint8_t)m;
            dfs(c, g + 1, m);
        } else if (f < c->fnext) {
            c->fnext = f;
        }
        c->t[np] = c->t[p];
        c->t[p] = 0;
        c->blank = p;
        if (c->stop)
            return;
    }
}

static void init_geometry(ctx_t *c, int W)
{
    c->W = W;
    c->N = W * W;
    for (int p = 0; p < c->N; ++p) {
        c->row[p] = p / W;
        c->col[p] = p % W;
    }
}

/* 1 if tiles is a permutation of 0..N-1 in the goal's parity class.
 * Sliding the blank horizontally changes neither the inversion count of the
 * non-blank tiles (read row-major) nor the blank's row; sliding it
 * vertically moves one tile past W-1 others (changing the inversion count by
 * an amount of the parity of W-1) and changes the blank's row by one. So for
 * odd W the inversion parity is invariant, and for even W the parity of
 * inversions + blank row is; the goal has 0 of both. */
int oracle_is_solvable(int W, const uint8_t *tiles)
{
    if (W < 2 || W > OR_MAX_W)
        return 0;
    int N = W * W;
    int seen[OR_MAX_N] = {0};
    int blank = -1;
    for (int p = 0; p < N; ++p) {
        int v = tiles[p];
        if (v >= N || seen[v])
            return 0;
        seen[v] = 1;
        if (v == 0)
            blank = p;
    }
    int inv = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] == 0)
            continue;
        for (int j = i + 1; j < N; ++j)
            if (tiles[j] != 0 && tiles[i] > tiles[j])
                inv++;
    }
    if (W % 2 == 1)
        return inv % 2 == 0;
    return (inv + blank / W) % 2 == 0;
}

int oracle_manhattan(int W, const uint8_t *tiles)
{
    ctx_t c;
    init_geometry(&c, W);
    memcpy(c.t, tiles, (size_t)c.N);
    return manhattan(&c);
}

/*
 * Solve one instance.
 *   count_all   1 = run the final iteration to completion (all optimal
 *               solutions counted), 0 = stop at the first goal popped.
 *   node_budget 0 = none; otherwise stop with OR_BUDGET once more nodes
 *               than this have been popped over all iterations.
 * Outputs (caller-allocated):
 *   out_moves[max_len]       first solution found (moves 0..3), zero-filled
 *   out_nodes[max_iters]     nodes popped per iteration, zero-filled
 *   out_limits[max_iters]    f-limit of each iteration, zero-filled
 *   *out_len, *out_iters, *out_solutions, *out_h0
 * Returns a status code.
 */
int oracle_ida(int W, const uint8_t *tiles, int count_all, uint64_t node_budget,
               int max_iters, int max_len, int *out_len, uint8_t *out_moves,
               uint64_t *out_nodes, int *out_limits, int *out_iters,
               uint64_t *out_solutions, int *out_h0)
{
    *out_len = -1;
    *out_iters = 0;
    *out_solutions = 0;
    *out_h0 = -1;
    if (max_len > 0)
        memset(out_moves, 0, (size_t)max_len);
    if (max_iters > 0) {
        memset(out_nodes, 0, sizeof(uint64_t) * (size_t)max_iters);
        memset(out_limits, 0, sizeof(int) * (size_t)max_iters);
    }
    if (W < 2 || W > OR_MAX_W || max_iters <= 0 || max_len <= 0 || max_len > OR_MAX_PATH)
        return OR_BADARG;
    if (!oracle_is_solvable(W, tiles))
        return OR_INVALID;

    ctx_t *c = (ctx_t *)calloc(1, sizeof(ctx_t));
    if (!c)
        return OR_BADARG;
    init_geometry(c, W);
    memcpy(c->t, tiles, (size_t)c->N);
    for (int p = 0; p < c->N; ++p)
        if (c->t[p] == 0)
            c->blank = p;
    c->count_all = count_all;
    c->budget = node_budget;

    int h0 = manhattan(c);
    *out_h0 = h0;
    c->limit = h0;
    int status = OR_LIMIT;
    for (int it = 0; it < max_iters; ++it) {
        if (c->limit > max_len)
            break;
        c->nodes_it = 0;
        c->fnext = INT_MAX;
        c->stop = 0;
        dfs(c, 0, -1);
        out_nodes[it] = c->nodes_it;
        out_limits[it] = c->limit;
        *out_iters = it + 1;
        if (c->budget_hit) {
            status = OR_BUDGET;
            break;
        }
        if (c->solutions > 0) {
            *out_len = c->limit;
            memcpy(out_moves, c->first, (size_t)c->limit);
            *out_solutions = c->solutions;
            status = OR_OK;
            break;
        }
        if (c->fnext == INT_MAX)
            break; /* nothing pruned and no goal: cannot happen for a valid board */
        c->limit = c->fnext;
    }
    free(c);
    return status;
}

/* ---- batch driver: independent instances over a pool of pthreads ---- */

typedef struct {
    int W, n, count_all, max_iters, max_len;
    uint64_t node_budget;
    const uint8_t *tiles;
    int *out_len;
    uint8_t *out_moves;
    uint64_t *out_nodes;
    int *out_limits;
    int *out_iters;
    uint64_t *out_solutions;
    int *out_h0;
    int *out_status;
    int next;
    pthread_mutex_t mu;
} batch_t;

static void *batch_worker(void *arg)
{
    batch_t *b = (batch_t *)arg;
    int N = b->W * b->W;
    for (;;) {
        pthread_mutex_lock(&b->mu);
        int i = b->next++;
        pthread_mutex_unlock(&b->mu);
        if (i >= b->n)
            break;
        b->out_status[i] = oracle_ida(
            b->W, b->tiles + (size_t)i * N, b->count_all, b->node_budget, b->max_iters,
            b->max_len, &b->out_len[i], b->out_moves + (size_t)i * b->max_len,
            b->out_nodes + (size_t)i * b->max_iters, b->out_limits + (size_t)i * b->max_iters,
            &b->out_iters[i], &b->out_solutions[i], &b->out_h0[i]);
    }
    return NULL;
}

int oracle_ida_batch(int W, const uint8_t *tiles, int n, int count_all, uint64_t node_budget,
                     int max_iters, int max_len, int nthreads, int *out_len, uint8_t *out_moves,
                     uint64_t *out_nodes, int *out_limits, int *out_iters,
                     uint64_t *out_solutions, int *out_h0, int *out_status)
{
    if (n < 0 || nthreads < 1)
        return OR_BADARG;
    batch_t b;
    memset(&b, 0, sizeof b);
    b.W = W;
    b.n = n;
    b.count_all = count_all;
    b.node_budget = node_budget;
    b.max_iters = max_iters;
    b.max_len = max_len;
    b.tiles = tiles;
    b.out_len = out_len;
    b.out_moves = out_moves;
    b.out_nodes = out_nodes;
    b.out_limits = out_limits;
    b.out_iters = out_iters;
    b.out_solutions = out_solutions;
    b.out_h0 = out_h0;
    b.out_status = out_status;
    pthread_mutex_init(&b.mu, NULL);
    if (nthreads > n)
        nthreads = n > 0 ? n : 1;
    pthread_t th[256];
    if (nthreads > 256)
        nthreads = 256;
    for (int i = 0; i < nthreads; ++i)
        pthread_create(&th[i], NULL, batch_worker, &b);
    for (int i = 0; i < nthreads; ++i)
        pthread_join(th[i], NULL);
    pthread_mutex_destroy(&b.mu);
    return OR_OK;
}

/* ---- batch helpers for exhaustive checks ---- */

void oracle_manhattan_batch(int W, const uint8_t *tiles, int n, int *out)
{
    int N = W * W;
    for (int i = 0; i < n; ++i)
        out[i] = oracle_manhattan(W, tiles + (size_t)i * N);
}

void oracle_is_solvable_batch(int W, const uint8_t *tiles, int n, int *out)
{
    int N = W * W;
    for (int i = 0; i < n; ++i)
        out[i] = oracle_is_solvable(W, tiles + (size_t)i * N);
}
