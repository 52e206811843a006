// Host-side pattern-database object shared by the solver (bpida.cu) and
// the table builder (bpida_pdb.cu). Not part of the C ABI: callers see an
// opaque bpida_pdb.
#pragma once
#include "bpida_device.cuh"

struct bpida_pdb {
    int dev = 0;                              // device the tables live on
    int width = 0;                            // 3 or 4
    int ng = 0;                               // groups
    int k[bp::PDB_MAX_GROUPS] = {};           // tiles per group
    unsigned long long table_bytes[bp::PDB_MAX_GROUPS] = {};
    int max_value[bp::PDB_MAX_GROUPS] = {};   // largest entry of each table
    unsigned long long id = 0;                // unique per object (keys cached graphs)
    unsigned char *tab = nullptr;             // all tables, one after another (device)
    bp::PdbInfo info = {};                    // layout (host copy)
    bp::PdbInfo *d_info = nullptr;            // layout (device copy)
    unsigned long long goal = 0;              // the goal's inverse board
    unsigned long long goal_sb = 0;           // the goal's slot board
};
