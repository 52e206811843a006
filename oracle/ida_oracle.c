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
 *
 * Second heuristic: additive disjoint pattern databases, the memory-
 * intensive heuristic that the paper's conclusion names as future work
 * (Section 7). See "pattern databases" below; the search itself is the
 * same, only h(t) changes. Parity status: pinned (an independent 0-1
 * breadth-first search of the abstract spaces, the reduction of singleton
 * groups to the Manhattan distance, admissibility and consistency on every
 * 8-puzzle edge, BFS lengths and path counts, and the tree-size recurrence
 * with the same heuristic).
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
    const struct heur *hp;  /* pattern databases; NULL = Manhattan distance */
} ctx_t;

/* ---- pattern databases ----
 * Tiles 1..N-1 are split into disjoint groups. For a group G with tiles
 * t_0 < ... < t_{k-1}, an abstract state is the positions of G's tiles and
 * of the blank (the other tiles are not told apart). An abstract move swaps
 * the blank with an adjacent cell; it costs 1 if that cell holds a tile of
 * G and 0 otherwise, so every real move is charged to exactly one group.
 * d_G(state) is the cost of a cheapest abstract path to the abstract goal
 * (tile t_j at position t_j, blank at 0), and h = sum over groups of d_G of
 * the board's abstraction: admissible because a real solution projects to
 * an abstract path in every group whose costs add up to its length, and
 * consistent because a real move changes one group's abstract state along
 * one edge (cost 1: d_G changes by at most 1) and every other group's along
 * a cost-0 edge (d_G unchanged). Keeping the blank in the abstract state is
 * what makes the second part hold. A cost-1 move shifts one tile of G by
 * one cell and a cost-0 move none, so d_G has the parity of the Manhattan
 * distance of G's tiles: h changes by exactly 1 per move, as the Manhattan
 * distance does, and the limits rise by exactly 2.
 * Table of group G: index = sum_j pos(t_j) << 4j | blank << 4k, 16^(k+1)
 * bytes, 255 where no abstract state has that index. */
#define OR_MAX_GROUPS 15
#define OR_MAX_GROUP_TILES 6
typedef struct heur {
    int ng;
    int k[OR_MAX_GROUPS];
    int tiles[OR_MAX_GROUPS][OR_MAX_GROUP_TILES];
    const uint8_t *tab[OR_MAX_GROUPS];
} heur_t;

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

/* h = sum over groups of the table entry of the board's abstraction. */
static int pdb_sum(const ctx_t *c)
{
    int pos[OR_MAX_N];
    for (int p = 0; p < c->N; ++p)
        pos[c->t[p]] = p;
    int h = 0;
    for (int g = 0; g < c->hp->ng; ++g) {
        uint64_t idx = 0;
        int k = c->hp->k[g];
        for (int j = 0; j < k; ++j)
            idx |= (uint64_t)pos[c->hp->tiles[g][j]] << (4 * j);
        idx |= (uint64_t)pos[0] << (4 * k);
        h += c->hp->tab[g][idx];
    }
    return h;
}

static int heuristic(const ctx_t *c)
{
    return c->hp ? pdb_sum(c) : manhattan(c);
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
        int f = g + 1 + heuristic(c);
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
static int ida_run(int W, const uint8_t *tiles, int count_all, uint64_t node_budget,
                   int max_iters, int max_len, const heur_t *hp, int *out_len, uint8_t *out_moves,
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
    c->hp = hp;

    int h0 = heuristic(c);
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

int oracle_ida(int W, const uint8_t *tiles, int count_all, uint64_t node_budget,
               int max_iters, int max_len, int *out_len, uint8_t *out_moves,
               uint64_t *out_nodes, int *out_limits, int *out_iters,
               uint64_t *out_solutions, int *out_h0)
{
    return ida_run(W, tiles, count_all, node_budget, max_iters, max_len, NULL, out_len, out_moves,
                   out_nodes, out_limits, out_iters, out_solutions, out_h0);
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
    const heur_t *hp;
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
        b->out_status[i] = ida_run(
            b->W, b->tiles + (size_t)i * N, b->count_all, b->node_budget, b->max_iters,
            b->max_len, b->hp, &b->out_len[i], b->out_moves + (size_t)i * b->max_len,
            b->out_nodes + (size_t)i * b->max_iters, b->out_limits + (size_t)i * b->max_iters,
            &b->out_iters[i], &b->out_solutions[i], &b->out_h0[i]);
    }
    return NULL;
}

static int ida_batch(int W, const uint8_t *tiles, int n, int count_all, uint64_t node_budget,
                     int max_iters, int max_len, int nthreads, const heur_t *hp, int *out_len,
                     uint8_t *out_moves, uint64_t *out_nodes, int *out_limits, int *out_iters,
                     uint64_t *out_solutions, int *out_h0, int *out_status)
{
    if (n < 0 || nthreads < 1)
        return OR_BADARG;
    batch_t b;
    memset(&b, 0, sizeof b);
    b.hp = hp;
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

int oracle_ida_batch(int W, const uint8_t *tiles, int n, int count_all, uint64_t node_budget,
                     int max_iters, int max_len, int nthreads, int *out_len, uint8_t *out_moves,
                     uint64_t *out_nodes, int *out_limits, int *out_iters,
                     uint64_t *out_solutions, int *out_h0, int *out_status)
{
    return ida_batch(W, tiles, n, count_all, node_budget, max_iters, max_len, nthreads, NULL, out_len,
                     out_moves, out_nodes, out_limits, out_iters, out_solutions, out_h0, out_status);
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

/* ---- pattern databases: construction and the searches that use them ---- */

/* Reads the groups: group_of_tile[t] is the group of tile t (t >= 1; entry
 * 0, the blank, is ignored); groups are numbered 0..ng-1 and each holds 1 to
 * OR_MAX_GROUP_TILES tiles, listed in increasing order. */
static int parse_groups(int W, const int *group_of_tile, heur_t *hp)
{
    memset(hp, 0, sizeof *hp);
    if (W < 2 || W > 4 || !group_of_tile)
        return OR_BADARG; /* positions take 4 bits in a table index */
    int N = W * W;
    for (int t = 1; t < N; ++t) {
        int g = group_of_tile[t];
        if (g < 0 || g >= OR_MAX_GROUPS || hp->k[g] >= OR_MAX_GROUP_TILES)
            return OR_BADARG;
        hp->tiles[g][hp->k[g]++] = t;
        if (g + 1 > hp->ng)
            hp->ng = g + 1;
    }
    for (int g = 0; g < hp->ng; ++g)
        if (hp->k[g] == 0)
            return OR_BADARG;
    return OR_OK;
}

uint64_t oracle_pdb_table_bytes(int k)
{
    return (k < 1 || k > OR_MAX_GROUP_TILES) ? 0 : (uint64_t)1 << (4 * (k + 1));
}

typedef struct {
    uint32_t *v;
    size_t n, cap;
} list_t;

static int list_push(list_t *l, uint32_t x)
{
    if (l->n == l->cap) {
        size_t nc = l->cap ? 2 * l->cap : 4096;
        uint32_t *p = (uint32_t *)realloc(l->v, nc * sizeof *p);
        if (!p)
            return 0;
        l->v = p;
        l->cap = nc;
    }
    l->v[l->n++] = x;
    return 1;
}

/* The tile slot j of abstract state s that sits at cell q, or -1. */
static int group_tile_at(uint32_t s, int k, int q)
{
    for (int j = 0; j < k; ++j)
        if ((int)((s >> (4 * j)) & 15u) == q)
            return j;
    return -1;
}

/*
 * Fills out (16^(k+1) bytes) with d_G for group `group`: a breadth-first
 * search from the abstract goal by cost layers (every abstract move is
 * reversible at the same cost, so distances from the goal are distances to
 * it). Layer d is first closed under cost-0 moves, then its cost-1
 * successors not yet reached form layer d + 1. *out_max = largest distance.
 */
int oracle_pdb_build(int W, const int *group_of_tile, int group, uint8_t *out, uint64_t out_bytes,
                     int *out_max)
{
    heur_t h;
    if (parse_groups(W, group_of_tile, &h) != OR_OK || group < 0 || group >= h.ng || !out)
        return OR_BADARG;
    const int k = h.k[group];
    const uint64_t size = oracle_pdb_table_bytes(k);
    if (out_bytes < size)
        return OR_BADARG;
    memset(out, 255, size);
    ctx_t geo;
    init_geometry(&geo, W);
    uint32_t goal = 0; /* tile t_j at position t_j, blank at 0 */
    for (int j = 0; j < k; ++j)
        goal |= (uint32_t)h.tiles[group][j] << (4 * j);
    const uint32_t blank_field = 15u << (4 * k);
    list_t cur = {0}, nxt = {0};
    int rc = OR_OK, d = 0, dmax = 0;
    out[goal] = 0;
    if (!list_push(&cur, goal))
        rc = OR_BADARG;
    while (rc == OR_OK && cur.n > 0) {
        /* cost 0: the blank moves into a cell without a tile of the group */
        for (size_t i = 0; i < cur.n && rc == OR_OK; ++i) {
            const uint32_t s = cur.v[i];
            const int blank = (int)((s >> (4 * k)) & 15u);
            for (int m = 0; m < 4; ++m) {
                const int nb = blank_target(&geo, blank, m);
                if (nb < 0 || group_tile_at(s, k, nb) >= 0)
                    continue;
                const uint32_t s2 = (s & ~blank_field) | ((uint32_t)nb << (4 * k));
                if (out[s2] == 255) {
                    out[s2] = (uint8_t)d;
                    if (!list_push(&cur, s2))
                        rc = OR_BADARG;
                }
            }
        }
        /* cost 1: the blank swaps with a tile of the group */
        nxt.n = 0;
        for (size_t i = 0; i < cur.n && rc == OR_OK; ++i) {
            const uint32_t s = cur.v[i];
            const int blank = (int)((s >> (4 * k)) & 15u);
            for (int m = 0; m < 4; ++m) {
                const int nb = blank_target(&geo, blank, m);
                const int j = nb < 0 ? -1 : group_tile_at(s, k, nb);
                if (j < 0)
                    continue;
                uint32_t s2 = s & ~blank_field & ~(15u << (4 * j));
                s2 |= ((uint32_t)blank << (4 * j)) | ((uint32_t)nb << (4 * k));
                if (out[s2] == 255) {
                    if (d + 1 > 254) {
                        rc = OR_LIMIT;
                        break;
                    }
                    out[s2] = (uint8_t)(d + 1);
                    dmax = d + 1;
                    if (!list_push(&nxt, s2))
                        rc = OR_BADARG;
                }
            }
        }
        list_t t = cur;
        cur = nxt;
        nxt = t;
        ++d;
    }
    free(cur.v);
    free(nxt.v);
    if (out_max)
        *out_max = dmax;
    return rc;
}

/* tables: the groups' tables one after another, in group order. */
static int make_heur(int W, const int *group_of_tile, const uint8_t *tables, heur_t *h)
{
    if (parse_groups(W, group_of_tile, h) != OR_OK || !tables)
        return OR_BADARG;
    uint64_t off = 0;
    for (int g = 0; g < h->ng; ++g) {
        h->tab[g] = tables + off;
        off += oracle_pdb_table_bytes(h->k[g]);
    }
    return OR_OK;
}

/* Heuristic value of each board (rows of W*W tiles). */
int oracle_pdb_h_batch(int W, const int *group_of_tile, const uint8_t *tables, const uint8_t *tiles, int n,
                       int *out)
{
    heur_t h;
    if (make_heur(W, group_of_tile, tables, &h) != OR_OK || n < 0)
        return OR_BADARG;
    ctx_t *c = (ctx_t *)calloc(1, sizeof(ctx_t));
    if (!c)
        return OR_BADARG;
    init_geometry(c, W);
    c->hp = &h;
    for (int i = 0; i < n; ++i) {
        memcpy(c->t, tiles + (size_t)i * c->N, (size_t)c->N);
        out[i] = heuristic(c);
    }
    free(c);
    return OR_OK;
}

/* oracle_ida_batch with the pattern-database heuristic. */
int oracle_ida_pdb_batch(int W, const int *group_of_tile, const uint8_t *tables, const uint8_t *tiles, int n,
                         int count_all, uint64_t node_budget, int max_iters, int max_len, int nthreads,
                         int *out_len, uint8_t *out_moves, uint64_t *out_nodes, int *out_limits,
                         int *out_iters, uint64_t *out_solutions, int *out_h0, int *out_status)
{
    heur_t h;
    if (make_heur(W, group_of_tile, tables, &h) != OR_OK)
        return OR_BADARG;
    return ida_batch(W, tiles, n, count_all, node_budget, max_iters, max_len, nthreads, &h, out_len, out_moves,
                     out_nodes, out_limits, out_iters, out_solutions, out_h0, out_status);
}
