// Internal layout of a selection (gc_sel) shared by the X-engine and the
// calibration translation units.
#pragma once

#include <vector>

#include "gc_internal.h"

#define GC_XENG_NTY 16   // types per X-engine work group

struct gc_sel {
    int scheme = 0;        // 0 subset, 1 low-cadence
    int L = 0, T = 0, P = 0, n_ubl = 0, n_cycle = 1, t_int = 0, null_dim = 0;
    double target = 0.0;
    std::vector<int32_t> types;      // [n_ubl][2] (dx, dy)
    std::vector<int32_t> type_ptr;   // [n_ubl + 1]
    std::vector<int32_t> pair_i, pair_j, pair_type;   // [P]
    std::vector<int32_t> win_t0, win_t1;              // [n_ubl]
    // neighbour table [2][n_ubl][N]: pair index with antenna i as i_p (0) or
    // as j_p (1), -1 if none; empty when it would exceed 16 M entries
    std::vector<int32_t> nbr;
    // X-engine work groups (types sharing a window, <= GC_XENG_NTY each)
    int n_groups = 0, n_windows = 0;
    std::vector<int32_t> grp_types;  // type indices, grouped
    std::vector<int32_t> grp_off;    // [n_groups + 1]
    std::vector<int32_t> grp_t0, grp_t1, grp_first, grp_win, grp_dymax;   // [n_groups]
    // arrays on a partly occupied lattice (gc_selection_subset_masked)
    int lattice = 0;                 // 0 square, 1 triangular
    int masked = 0;                  // 1: only the points of `mask` hold antennas
    int n_occ = 0;                   // antennas (L * L when unmasked)
    std::vector<int32_t> mask;       // [L * L] 0 / 1 (masked only)
    // start-point tree over the (1,0) and (0,1) types (masked only), in
    // breadth-first order: antenna, the pair linking it to its parent (-1 for
    // the root) and +1 / -1 when the antenna is that pair's first / second member
    std::vector<int32_t> tree_ant, tree_pair, tree_sign;
    // device copies (one allocation, on `device`)
    int device = -1;
    void *d_base = nullptr;
    int32_t *d_types = nullptr, *d_type_ptr = nullptr, *d_pair_i = nullptr, *d_pair_j = nullptr,
            *d_pair_type = nullptr, *d_win_t0 = nullptr, *d_win_t1 = nullptr, *d_grp_types = nullptr,
            *d_grp_off = nullptr, *d_grp_t0 = nullptr, *d_grp_t1 = nullptr, *d_grp_first = nullptr,
            *d_grp_win = nullptr, *d_nbr = nullptr, *d_grp_dymax = nullptr, *d_mask = nullptr,
            *d_tree_ant = nullptr, *d_tree_pair = nullptr, *d_tree_sign = nullptr;
};

gc_status gc_sel_upload(gc_ctx *ctx, gc_sel *s);
void gc_sel_release_device(gc_sel *s);

// tensor-core X-engine (gc_xengine_tc.cu)
bool gc_xeng_tc_eligible(const gc_sel *sel, int vfmt, const void *volt, int L);
int gc_xeng_tc_slices(const gc_ctx *ctx, const gc_sel *sel, int L, int C);
gc_status gc_xeng_tc_launch(gc_ctx *ctx, const void *volt, int L, int C, int T, const gc_sel *sel, void *part,
                            void *apart, int n_tsplit, cudaStream_t s);
