// plan.h -- symbolic analysis of the sector pattern (host, once per L) and its device mirror.
//
// The pattern of H - sigma I does not depend on the fields, the seed or sigma, so one plan
// serves every factorization at a given L.  It holds the fill-reducing order, the supernodal
// assembly tree, the front row lists, the maps that scatter the CSR entries and the children's
// contribution blocks into the fronts, and the static launch schedule (levels x panels) that the
// batched numeric factorization and the triangular solves replay.
#pragma once

#include <utility>

#include "mbl_internal.h"

namespace mbl {

constexpr int NB = 64;  // panel width of the blocked frontal LDL^T (pivot window)
constexpr int RB = 64;  // rows per row block (stage 2 / solve updates)
constexpr int TB = 64;  // tile edge of the trailing (Schur) update
constexpr int ACOLS = 32;  // columns per assembly work item
constexpr int SPW = 256;   // width of a solve panel (4 factor panels): one dense block operator M each
constexpr int SUBS = SPW / NB;
constexpr int64_t ARENA_ALIGN = (int64_t)1 << 19;  // elements: 2 MiB in FP32, 4 MiB in FP64
constexpr int64_t LEAN_CHUNK = (int64_t)1 << 23;   // elements per physical chunk of the memory-lean arena

// One active front in one (level, panel) step.
struct PanelDesc {
    int32_t front;   // supernode id
    int32_t k0;      // first column of the panel inside the front
    int32_t w;       // panel width (<= NB)
    int32_t m2;      // rows below the diagonal block: f - k0 - w
    int64_t off2;    // prefix count of row blocks (stage 2) before this descriptor in its step
    int64_t off3;    // prefix count of trailing tiles (stage 3) before this descriptor in its step
    int64_t woff;    // offset (elements) of this front's W21 scratch (m2 x NB column-major, ld m2)
    int64_t off3t;   // prefix count of 128 x 128 tensor-core tiles before this descriptor in its step
};

struct PanelStep {
    int32_t level, kk;
    int32_t d0, nd;  // descriptor range
    int64_t n2, n3;  // row blocks and trailing tiles in this step
    int64_t n3t;     // 128 x 128 tensor-core tiles in this step
    int64_t wsize;   // W21 scratch elements used by this step
};

constexpr int RBF = 32;  // rows per CTA of a forward solve step
constexpr int RBB = 64;   // columns per chunk of a backward solve step; rows per CTA of the G = [M; L21 M] build
constexpr int RBK = 256;  // rows per CTA of a backward solve step

// One solve panel: columns [k0, k0 + w) of a front's fully-summed block (w <= SPW).  M (w x w) is
// the composite of the factor panels' pivot permutations and unit-lower eliminations restricted
// to the panel.  Once the factorization is done the panel's column block [k0, f) x [k0, k0 + w)
// holds G = [M; L21 M], so that the forward step is z_panel <- M z_panel, z_below -= (L21 M) z_panel
// (with z_panel read before the update) and the backward step is x_panel <- G^T [y_panel; -x_below].
struct SolveDesc {
    int32_t front, k0, w, m2;        // m2 = f - k0 - w rows below
    int64_t off;                     // prefix of forward row blocks (RBF rows of [k0, f)) in the step
    int64_t offb;                    // prefix of RBB-row tiles of [k0, f) in the step (G build)
    int64_t offk;                    // prefix of backward row blocks (RBK rows of [k0, f)) in the step
    int64_t moff;                    // offset (elements) of M while it is built
    int64_t goff;                    // offset (elements) of G in the packed solve factor
    int64_t offk_l;                  // prefix of backward-start row blocks within the level (level-wide launch)
    int32_t fdesc[SUBS];             // factor descriptors of the sub-panels (-1 if absent)
};

// Leading dimension of a panel's G (rows [k0, f) of the front) in the packed solve factor: rows
// padded to a multiple of 4 elements, so that every column starts on a 16-byte boundary; the
// padding rows are zero.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t sg_ld(int64_t rows) { return (rows + 3) & ~(int64_t)3; }

struct SolveStep {
    int32_t level;
    int32_t d0, nd;
    int64_t nrb;                     // forward row blocks in this step
    int64_t nrbb;                    // RBB-row tiles in this step
    int64_t nrbk;                    // backward row blocks in this step
    int32_t maxw;                    // widest panel of the step (backward column chunks = ceil(maxw / RBB))
    int64_t fblk0, bblk0;            // first entries of the step in fblk_desc / bblk_desc
};

// Row blocks of a panel in the backward start: block 0 holds the panel's own w rows; the others cover
// the contribution block from its first row (rounded down to 16 bytes) in RBK-row blocks; the rows of
// the front's later panels are left to the updates.  cb0 = nc - k0 (first contribution row, relative).
#ifdef __CUDACC__
__host__ __device__
#endif
inline int bwd_start_blocks(int R, int cb0) { return cb0 >= R ? 1 : 1 + (R - (cb0 & ~3) + RBK - 1) / RBK; }

// Backward sweep, level by level: one launch over every panel of the level starts each panel's
// accumulator acc_i = G_i^T [y_i; 0; -x_cb] (its own rows and the contribution block, whose x the
// ancestors have fixed); then, for j = K-1 .. 1 (K panels in the level's widest front), one launch
// subtracts G_i[rows of panel j]^T x_j from acc_i for every earlier panel i < j of every front with
// more than j panels (x_j = acc_j is final by then).  BwdUpd lists the (i, j) pairs of one launch.
struct BwdUpd {
    int32_t level, j;
    int64_t it0, nit;                // items bu_items[it0 .. it0 + nit): (descriptor of i, descriptor of j)
};

// Work item of the dataflow (persistent) solve: kind 0 = gather of rows [GR a, GR a + GR) of a
// front; kind 1 = panel step: solve descriptor a, row block b (RBF rows forward, RBK rows backward),
// column chunk cc (backward only).  Item lists are in a topological order of their dependencies.
constexpr int GR = 64;  // rows per gather item
struct SolveItem {
    int16_t kind, cc;
    int32_t front, a, b;
};

// Fronts [fo0, fo1) of one level whose contribution blocks are last read by the assembly of level
// `release` (their parents' level; the level itself for roots).
struct ArenaRegion {
    int32_t level, release;
    int64_t fo0, fo1;
};

struct AsmItem {     // assembly work item: columns [c0, c0 + ACOLS) of a front
    int32_t front, c0;
};

// Size classes of a panel step's largest trailing block m2 for the Schur-update autotuning:
// class c holds 64 2^c <= m2 < 64 2^(c+1) (class 0 also everything smaller, the last class everything
// larger).
constexpr int TUNE_CLASSES = 8;
inline int tune_class(int64_t m2) {
    int c = 0;
    while (c + 1 < TUNE_CLASSES && m2 >= ((int64_t)64 << (c + 1))) ++c;
    return c;
}

struct Plan {
    int L = 0;
    // Schur-update autotuning by tensor-core mode (1: 3xTF32, 2: 3xBF16) and size class: 1 = tcgen05
    // tiles, 0 = CUDA-core tiles; the timings (microseconds per update of the class's synthetic front,
    // tensor then CUDA cores, 0 where the class has no step) are kept for reporting.
    std::mutex tune_mu;
    bool tuned[3] = {};
    int8_t tune_tc[3][TUNE_CLASSES] = {};
    float tune_us[3][TUNE_CLASSES][2] = {};
    std::vector<int32_t> step_class;  // per panel step: class of its largest trailing block
    int64_t n = 0, nnzA = 0;
    std::vector<int32_t> perm, iperm;  // new -> old, old -> new
    int32_t ns = 0;
    std::vector<int32_t> sn_start, sn_nc, sn_f, sn_parent, sn_level;
    std::vector<int64_t> sn_rows_off, sn_fo, sn_zo, sn_rel_off;
    std::vector<int32_t> rows, relind;
    std::vector<int32_t> ch_ptr, ch_list;
    std::vector<int32_t> col_snode;           // new column -> supernode
    std::vector<int64_t> amap_ptr;            // new column -> entries (n + 1)
    std::vector<int64_t> amap_src;            // CSR position
    std::vector<int32_t> amap_row;            // local row in the front
    std::vector<int32_t> lvl_ptr, lvl_fronts;  // fronts by level
    // the fronts arena as regions of fronts sharing (level, release level), ordered by both; each
    // starts on an ARENA_ALIGN boundary.  lean_peak_elems is the most the regions hold at one time
    // when each is mapped from its level's assembly to its release.
    std::vector<ArenaRegion> regions;
    int64_t lean_peak_elems = 0;
    // (region, chunk) pairs lying wholly in one front's fully summed columns, by level (ptr nlevels + 1)
    std::vector<int64_t> lean_prefix_ptr;
    std::vector<std::pair<int32_t, int32_t>> lean_prefix;
    std::vector<int32_t> asm_ptr;             // assembly items by level
    std::vector<AsmItem> asm_items;
    std::vector<PanelStep> steps;
    std::vector<int32_t> lvl_step_ptr;        // steps by level
    std::vector<PanelDesc> descs;
    std::vector<SolveStep> ssteps;
    std::vector<int32_t> lvl_sstep_ptr;       // solve steps by level
    std::vector<SolveDesc> sdescs;
    // per forward (RBF rows) and backward (RBK rows) row block of each solve step, the index of its
    // descriptor within the step: one load instead of a search
    std::vector<int32_t> fblk_desc, bblk_desc;
    // level-wide backward start: per level its first descriptor, count, widest panel, row blocks and
    // block -> descriptor table (relative to the level's first descriptor, offsets in lvl_bblk0)
    std::vector<int32_t> lvl_d0, lvl_nd, lvl_maxw, lvl_maxr;  // maxr: most rows of a panel's G
    std::vector<int64_t> lvl_nrbk, lvl_bblk0;
    std::vector<int32_t> lvl_bblk_desc;
    int64_t max_lvl_nrbk = 0;
    // backward updates: per level, launches in order (bu_ptr by level), items as descriptor pairs
    std::vector<BwdUpd> bupd;
    std::vector<int32_t> bu_ptr;
    std::vector<int32_t> bu_items;   // 2 per item
    // forward-solve gather as row lists: for every row of every front of a level (levels in order),
    // its work row in Z, its own right-hand-side row (-1 below the fully summed block) and the Z
    // rows of the children's contribution blocks that land on it (children in tree order)
    std::vector<int64_t> lvl_fg_ptr;          // rows by level (nlevels + 1)
    std::vector<int64_t> fg_dst, fg_own, fg_cptr, fg_src;
    // dataflow solve: item lists and completion targets.  Per front: gather items, forward blocks
    // over all panels, backward (panel, column chunk) reductions over all panels, first fg row; per
    // solve descriptor: forward blocks of the front's earlier panels, backward chunks of its later
    // panels, and its first slot in the global backward-partials buffer.
    std::vector<SolveItem> df_fwd, df_bwd;
    std::vector<int32_t> df_gchunks, df_ftotal, df_btotal, df_fprefix, df_bprefix;
    std::vector<int64_t> df_fg_off, df_poff;
    int64_t df_pslots = 0;
    int64_t m_elems = 0, max_sstep_nrbb = 0, max_sstep_nrbk = 0;
    int64_t sg_elems = 0;                     // packed solve factor (all panels' G, padded columns)
    int64_t arena_elems = 0, zwork_elems = 0, wscratch_elems = 0, max_desc_per_step = 0;
    int64_t max_step_n2 = 0;
    int64_t nnz_l = 0;
    double flops = 0.0;
    int32_t max_front = 0, nlevels = 0;
    double ms_analyse = 0.0;
    int ordering = MBL_ORDER_BAND;  // the separator rule the ordering used

    // device mirror
    DVec<int32_t> d_perm, d_iperm, d_sn_start, d_sn_nc, d_sn_f, d_rows, d_relind, d_ch_ptr, d_ch_list, d_amap_row;
    DVec<int32_t> d_sn_parent;
    DVec<int64_t> d_sn_rows_off, d_sn_fo, d_sn_zo, d_sn_rel_off, d_amap_ptr, d_amap_src;
    DVec<AsmItem> d_asm_items;
    DVec<PanelDesc> d_descs;
    DVec<SolveDesc> d_sdescs;
    DVec<int32_t> d_fblk_desc, d_bblk_desc, d_lvl_bblk_desc, d_bu_items;
    DVec<int64_t> d_fg_dst, d_fg_own, d_fg_cptr, d_fg_src;
    DVec<SolveItem> d_df_fwd, d_df_bwd;
    DVec<int32_t> d_df_gchunks, d_df_ftotal, d_df_btotal, d_df_fprefix, d_df_bprefix;
    DVec<int64_t> d_df_fg_off, d_df_poff;
    bool on_device = false;
};

// Build the plan for the pattern of a sector (host arrays: states, rowptr, col of the CSR) with
// the fill-reducing ordering MBL_ORDER_* (MBL_ORDER_AUTO resolved by the sector dimension).
std::shared_ptr<Plan> build_plan(int L, const std::vector<uint32_t> &states, const std::vector<int64_t> &rowptr,
                                 const std::vector<int32_t> &col, int ordering = MBL_ORDER_AUTO);
void upload_plan(Ctx *ctx, Plan &p);

}  // namespace mbl
