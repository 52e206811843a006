// Pattern databases for the search (the memory-intensive heuristic that the
// paper's conclusion names as future work, Section 7): each group's table is
// built on the device by a breadth-first search of the group's abstract
// space, one cost layer at a time, and stays in device memory for the solve
// calls that use it (bpida_solve_pdb).
//
// Abstract space of a group G (k tiles): the positions of G's tiles and of
// the blank. The blank swaps with an adjacent cell; the move costs 1 if the
// cell holds a tile of G and 0 otherwise. Entry (index sum_j pos(t_j) << 4j |
// blank << 4k) = cost of a cheapest path to the abstract goal (tile t at cell
// t, blank at 0); moves are reversible at equal cost, so the search starts at
// the goal. Layer d is first closed under cost-0 moves (k_pdb_close: the
// blank's whole region, the cells it reaches without crossing a tile of G,
// takes distance d), then its cost-1 successors not yet reached take d + 1
// (k_pdb_expand). Every write of a launch stores the same value into an
// entry that was unreached (255), so the tables do not depend on the order
// in which threads run.
#include "bpida.h"
#include "bpida_pdb.h"

#include <atomic>
#include <cstdio>
#include <cstring>

using namespace bp;

namespace {

std::atomic<unsigned long long> g_pdb_ids{0};

// Cells whose column is not 0 / not W - 1 (targets of a shift right / left
// that did not wrap around a row end).
template <int W> __host__ __device__ constexpr uint32_t not_col(int c)
{
    uint32_t m = 0;
    for (int p = 0; p < W * W; ++p)
        if (p % W != c)
            m |= 1u << p;
    return m;
}

template <int W>
__global__ void k_pdb_close(unsigned char *tab, int k, unsigned long long size, int d)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= size || tab[i] != (unsigned char)d)
        return;
    const int kb = 4 * k;
    uint32_t occ = 0;
    for (int j = 0; j < k; ++j)
        occ |= 1u << ((i >> (4 * j)) & 15u);
    const int blank = (int)((i >> kb) & 15u);
    const uint32_t free_cells = ((1u << (W * W)) - 1u) & ~occ;
    uint32_t region = 1u << blank;
    for (int it = 0; it < W * W; ++it) {
        const uint32_t g = (region | ((region << 1) & not_col<W>(0)) | ((region >> 1) & not_col<W>(W - 1)) |
                            (region << W) | (region >> W)) &
                           free_cells;
        if (g == region)
            break;
        region = g;
    }
    const unsigned long long rest = i & ~(15ull << kb);
    for (uint32_t r = region & ~(1u << blank); r; r &= r - 1u) {
        unsigned char *e = tab + (rest | ((unsigned long long)(__ffs((int)r) - 1) << kb));
        if (*e == 255)
            *e = (unsigned char)d;
    }
}

template <int W>
__global__ void k_pdb_expand(unsigned char *tab, int k, unsigned long long size, int d, unsigned long long *added)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= size || tab[i] != (unsigned char)d)
        return;
    const int kb = 4 * k;
    const int blank = (int)((i >> kb) & 15u);
    const int r = blank / W, c = blank % W;
    unsigned n = 0;
    for (int m = 0; m < 4; ++m) {
        const int nb = m == 0 ? (r > 0 ? blank - W : -1)
                     : m == 1 ? (c > 0 ? blank - 1 : -1)
                     : m == 2 ? (c < W - 1 ? blank + 1 : -1)
                              : (r < W - 1 ? blank + W : -1);
        if (nb < 0)
            continue;
        int j = -1;
        for (int q = 0; q < k; ++q)
            if ((int)((i >> (4 * q)) & 15u) == nb)
                j = q;
        if (j < 0)
            continue;
        // the tile moves into the blank's cell, the blank to nb
        const unsigned long long i2 = (i & ~(15ull << kb) & ~(15ull << (4 * j))) |
                                      ((unsigned long long)blank << (4 * j)) | ((unsigned long long)nb << kb);
        if (tab[i2] == 255) {
            tab[i2] = (unsigned char)(d + 1);
            ++n;
        }
    }
    if (n)
        atomicAdd(added, (unsigned long long)n);
}

template <int W>
bpida_status build_tables(bpida_pdb &P, const int tiles[][PDB_MAX_TILES], cudaStream_t st)
{
    unsigned long long *d_added = nullptr, h_added = 0;
    if (cudaMalloc(&d_added, sizeof *d_added) != cudaSuccess)
        return BPIDA_ENOMEM;
    bpida_status rc = BPIDA_OK;
    unsigned long long off = 0;
    for (int g = 0; g < P.ng && rc == BPIDA_OK; ++g) {
        const int k = P.k[g];
        const unsigned long long size = P.table_bytes[g];
        unsigned char *tab = P.tab + off;
        off += size;
        unsigned long long goal = 0;  // tile t_j at cell t_j, blank at 0
        for (int j = 0; j < k; ++j)
            goal |= (unsigned long long)tiles[g][j] << (4 * j);
        if (cudaMemsetAsync(tab, 255, size, st) != cudaSuccess || cudaMemsetAsync(tab + goal, 0, 1, st) != cudaSuccess) {
            rc = BPIDA_ECUDA;
            break;
        }
        const unsigned blocks = (unsigned)((size + 255) / 256);
        for (int d = 0;; ++d) {
            if (d >= 254) {
                rc = BPIDA_ELIMIT;  // a distance that does not fit a table byte
                break;
            }
            k_pdb_close<W><<<blocks, 256, 0, st>>>(tab, k, size, d);
            cudaMemsetAsync(d_added, 0, sizeof *d_added, st);
            k_pdb_expand<W><<<blocks, 256, 0, st>>>(tab, k, size, d, d_added);
            if (cudaMemcpyAsync(&h_added, d_added, sizeof h_added, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = BPIDA_ECUDA;
                break;
            }
            if (h_added == 0) {
                P.max_value[g] = d;
                break;
            }
        }
    }
    cudaFree(d_added);
    return rc;
}

}  // namespace

extern "C" {

bpida_status bpida_pdb_create(int width, const int *group_of_tile, bpida_pdb **out, void *stream)
{
    if (!out)
        return BPIDA_EINVAL;
    *out = nullptr;
    if ((width != 3 && width != 4) || !group_of_tile)
        return BPIDA_EINVAL;
    const int N = width * width;
    bpida_pdb P;
    int tiles[PDB_MAX_GROUPS][PDB_MAX_TILES];
    for (int t = 1; t < N; ++t) {
        const int g = group_of_tile[t];
        if (g < 0 || g >= PDB_MAX_GROUPS || P.k[g] >= PDB_MAX_TILES)
            return BPIDA_EINVAL;
        tiles[g][P.k[g]++] = t;
        P.ng = g + 1 > P.ng ? g + 1 : P.ng;
    }
    for (int g = 0; g < P.ng; ++g)
        if (P.k[g] == 0)
            return BPIDA_EINVAL;
    P.width = width;
    if (cudaGetDevice(&P.dev) != cudaSuccess)
        return BPIDA_ECUDA;

    // layout: slot 0 the blank, then each group's tiles in increasing order
    std::memset(&P.info, 0, sizeof P.info);
    P.info.ng = P.ng;
    int slot = 1;
    unsigned long long base = 0;
    for (int g = 0; g < P.ng; ++g) {
        P.table_bytes[g] = 1ull << (4 * (P.k[g] + 1));
        P.info.goff[g] = 4 * slot;
        P.info.gbits[g] = 4 * P.k[g];
        P.info.base[g] = (unsigned)base;
        for (int j = 0; j < P.k[g]; ++j, ++slot) {
            const int t = tiles[g][j];
            P.info.slot_of_tile[t] = (unsigned char)slot;
            P.info.tile_of_slot[slot] = (unsigned char)t;
            P.info.slot[slot].goff = (unsigned)P.info.goff[g];
            P.info.slot[slot].mask = (1u << P.info.gbits[g]) - 1u;
            P.info.slot[slot].vsh = (unsigned)(PDB_VSHIFT + 2 * g);
            P.info.slot[slot].base = (unsigned)base;
            // tile t's goal cell is t: inverse field `slot` = t, slot-board field t = slot
            P.goal |= (unsigned long long)t << (4 * slot);
            P.goal_sb |= (unsigned long long)slot << (4 * t);
        }
        base += P.table_bytes[g];
    }
    if (base >= (1ull << 32))
        return BPIDA_EINVAL;

    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMalloc(&P.tab, base) != cudaSuccess) {
        cudaGetLastError();
        return BPIDA_ENOMEM;
    }
    if (cudaMalloc(&P.d_info, sizeof(PdbInfo)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(P.tab);
        return BPIDA_ENOMEM;
    }
    bpida_status rc = width == 3 ? build_tables<3>(P, tiles, st) : build_tables<4>(P, tiles, st);
    if (rc == BPIDA_OK &&
        (cudaMemcpyAsync(P.d_info, &P.info, sizeof(PdbInfo), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        rc = BPIDA_ECUDA;
    if (rc == BPIDA_OK && cudaGetLastError() != cudaSuccess)
        rc = BPIDA_ECUDA;
    if (rc != BPIDA_OK) {
        cudaFree(P.tab);
        cudaFree(P.d_info);
        return rc;
    }
    P.id = ++g_pdb_ids;
    *out = new bpida_pdb(P);
    return BPIDA_OK;
}

void bpida_pdb_destroy(bpida_pdb *pdb)
{
    if (!pdb)
        return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(pdb->dev);
    // solve calls are asynchronous: one that reads the tables may still run
    cudaDeviceSynchronize();
    cudaFree(pdb->tab);
    cudaFree(pdb->d_info);
    cudaSetDevice(cur);
    delete pdb;
}

int bpida_pdb_groups(const bpida_pdb *pdb) { return pdb ? pdb->ng : 0; }

uint64_t bpida_pdb_table_bytes(const bpida_pdb *pdb, int group)
{
    return (pdb && group >= 0 && group < pdb->ng) ? pdb->table_bytes[group] : 0;
}

int bpida_pdb_max_value(const bpida_pdb *pdb, int group)
{
    return (pdb && group >= 0 && group < pdb->ng) ? pdb->max_value[group] : -1;
}

bpida_status bpida_pdb_copy_table(const bpida_pdb *pdb, int group, uint8_t *dst, uint64_t bytes, void *stream)
{
    if (!pdb || group < 0 || group >= pdb->ng || !dst || bytes < pdb->table_bytes[group])
        return BPIDA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dst, pdb->tab + pdb->info.base[group], pdb->table_bytes[group], cudaMemcpyDefault, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BPIDA_ECUDA;
    return BPIDA_OK;
}

}  // extern "C"
