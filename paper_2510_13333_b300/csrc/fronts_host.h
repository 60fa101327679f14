#pragma once

#include "internal.h"

namespace scopf {

// Host copy of the frontal structure (see kernels.h: DevFront).
struct HostFronts {
    int n_tasks = 0, n_blocks = 0, n_border = 0, max_level = 0, n_small = 0;
    std::vector<int64_t> front_off, vec_off, rows_off, rel_off, border_off, border_vec_off, scatter;
    std::vector<int32_t> f, npiv, parent, is_border, child_ptr, child, rel, level, block;
    std::vector<int64_t> rows, border_rows, orig_ptr, orig_nz;
    std::vector<int32_t> orig_off;
    // work items: contiguous task ranges (a subtree of small fronts run by
    // one warp in postorder, or a single front) and their tree
    int n_items = 0, n_items_small = 0, n_items_med = 0;
    std::vector<int32_t> item_ptr, item_of_task, item_parent, item_is_border, item_child_ptr,
        item_child, item_cont;
    // ready-queue seeds: items runnable at the start of each sweep, and the
    // dependency counts the sweeps start from
    std::vector<int32_t> init_small, init_med, init_big, init_fwd, init_bwd, pend_factor, nchild;
    // packed records (see kernels.h: DevFront::task_rec, child_rec)
    std::vector<int32_t> task_rec, child_rec;
    std::vector<int64_t> vpos_of_row;   // per KKT row: vector slot of its pivot, -1 border
    int64_t front_elems = 0, vec_elems = 0, nnz_L = 0;
    double flops = 0;
};

std::string build_fronts(const Model &M, const std::vector<BlockSymbolic> &syms, int cluster_cap,
                         HostFronts &H);

}  // namespace scopf
