// Host-side symbolic setup of the multi-area Gauss-Newton pipeline.
//
// One-time analysis (Sec. 4.1 "one-time symbolic dependency analysis",
// Sec. 4.3 "CSR sparsity pattern is constructed once"): boundary sets and
// selectors E_k (Sec. 2.3, Eq. Ek_select), fixed measurement templates in
// structure-of-arrays form, slot maps that send every gain-matrix term to its
// place in the factor storage (Sec. 4.2), and supernodal symbolic factors
// with a trailing dense Schur block (Sec. 4.3) for every area and for the
// boundary system (Sec. 4.4).  Nothing here touches the GPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace mase {

// Supernodal symbolic Cholesky factor of an SPD system whose last n_bnd
// scalar unknowns are not eliminated: after factoring the first n_int columns
// the trailing block holds the Schur complement (Eq. schur_defs).
//
// Storage (element offsets): supernode s owns a dense column-major block of
// ld_s = w_s + nr_s rows by w_s columns at sn_off[s]; rows 0..w_s-1 are its
// diagonal block (lower part used), rows w_s.. are its off-diagonal row set
// R_s (rows[sn_rows[s] ...], sorted scalar indices).  The Schur block is
// stored packed lower, column-major, at off_B.  After the numeric
// factorisation the diagonal entries hold 1/L_cc.
struct SymFactor {
    int n_int = 0, n_bnd = 0;
    std::vector<int> sn_c0, sn_w, sn_nr, sn_off, sn_rows;
    std::vector<int> rows;               // concatenated R_s
    std::vector<int> colbase, relbase;   // per R_s entry: target column base, rel index base
    std::vector<int> rel;                // relative row positions in target supernodes
    std::vector<int> lev_off;            // supernodes of level l: sn_order[lev_off[l]..lev_off[l+1])
    std::vector<int> sn_order;
    std::vector<int> lev_items;          // per level: update items (pairs + rhs rows)
    // column units of the update phase: unit u covers target columns
    // unit_j[u] .. unit_j[u] + unit_nj[u] (at most kUnitCols) of supernode
    // unit_sn[u]'s row set, all in one target segment (they share the
    // relative-index array); units of level l are [lev_units[l], lev_units[l+1])
    std::vector<int> unit_sn, unit_j, unit_nj, lev_units;
    // dataflow task records of the numeric factorisation, 16 ints each:
    // {type << 24 | s, wait counter, wait threshold, counter to signal or -1},
    // then per type
    //   D (0): {sn_off, w, ld, c0}
    //   C (1): {sn_off, w, ld, r0}
    //   U (2): {sn_off + w, relbase, sn_rows, c0}, {w | nj << 8, ld | j0 << 16,
    //          rhs end (0: no rhs rows), colbase 0}, {colbase 1..3, 0}
    // counters: [0, nsn) updates received by supernode t, [nsn, 2 nsn)
    // diagonal block and panel chunks finished for supernode s
    std::vector<int> tasks;
    int n_tasks = 0;
    // level schedule instead of dataflow: level l runs tasks
    // [lev_tasks[3l], lev_tasks[3l+1]) (D), then [.., lev_tasks[3l+2]) (C),
    // then [.., lev_tasks[3l+3]) (U), with a block barrier after each group
    int level_sched = 0;
    std::vector<int> lev_tasks;
    double sched_cycles = 0.0;           // estimated makespan of the task order
    // row chunks of the panels below their diagonal blocks: level l owns
    // records [lev_chunks[l], lev_chunks[l+1]), 8 ints each
    // {sn_off, w, ld, r0, c0, sn_rows, 0, 0}
    std::vector<int> chunk_rec, lev_chunks;

    std::vector<int> var_sn;             // internal scalar var -> supernode
    int store_int = 0, off_B = 0, store_total = 0;
    int max_w = 0;
    long long flops = 0;                 // multiply-adds of one numeric factorisation
    long long pairs = 0;

    int nsn() const { return (int)sn_c0.size(); }
    int nlev() const { return (int)lev_items.size(); }
    // storage offset of lower entry (r, c), r >= c; -1 if outside the pattern
    int pos(int r, int c) const;
};

// Widest supernode panel, in scalar columns: one warp factors a diagonal block
// of at most this width (wider than 16 as 2 x 2 blocks of 16).  Area factors
// run as a dataflow whose critical path grows with the panel width, so they
// use narrower panels than the level-scheduled boundary factor.
constexpr int kMaxPanel = 32;
constexpr int kAreaPanel = 16;
constexpr int kBoundaryPanel = 32;
// Target columns handled together by one update unit.
constexpr int kUnitCols = 4;
// Warps the task order is scheduled for (512-thread blocks).
constexpr int kTaskWarps = 16;

// builds F.tasks (needs the units, chunks and update maps of F): a list
// schedule for the dataflow, or (level_sched) level by level with the
// diagonal blocks, panel chunks and units of each level in F.lev_tasks
void build_tasks(SymFactor &F, int nwarps, bool level_sched);

// Bus-level system: nodes [0, nb_int) are eliminated in a fill-reducing
// order, nodes [nb_int, nb_int + nb_bnd) are kept (in the given order).
struct BusSystem {
    int nb_int = 0, nb_bnd = 0;
    std::vector<std::vector<int>> adj;   // symmetric, no self loops
    std::vector<int> nvar;               // 1 (slack: magnitude only) or 2
};

struct SymResult {
    std::vector<int> order;   // position -> node
    std::vector<int> pos_of;  // node -> position
    std::vector<int> var0;    // position -> first scalar unknown (size npos+1)
    SymFactor F;
};

// Exact minimum-degree ordering of the internal nodes on the elimination
// graph, fundamental supernodes, level schedule and update maps.
// relax_alpha bounds the explicit zeros a merge may add (fraction of the
// merged panel), relax_wmax the merged width in buses; 0 gives fundamental
// supernodes only.
SymResult build_symbolic(const BusSystem &sys, double relax_alpha = 0.30, int relax_wmax = 16,
                         int max_panel = kAreaPanel, bool level_sched = false);

// Dynamic shared-memory layout of the area kernel for one area (byte
// offsets, 16-byte aligned): FP64 gradient, rhs in the solve type, bus
// magnitude/cos/sin (FP64), per-end buffer (flows, then gain partials),
// per-bus weighted injection residuals, per-bus injection self partials, and
// the factor storage when it fits.
struct SmemLayout {
    size_t off_g, off_y, off_bus, off_end, off_inj, off_self, off_st, vector_bytes;
};
SmemLayout area_smem_layout(int nv, int nb_loc, int n_ends, int n_own, size_t rg, size_t rs);

// Shared memory one block may use on the target GPU (227 KB opt-in less 1 KB
// of static shared memory).
constexpr int kDefaultSmemLimit = 227 * 1024 - 1024;

// ---------------------------------------------------------------------------
// Complete problem setup
// ---------------------------------------------------------------------------
struct NetIn {
    int n_bus, n_branch, slack;
    const int32_t *from, *to;
    const double *r, *x, *bc;
};

struct AreaSetup {
    int k;
    int nb_int, nb_loc;                  // internal buses, local buses (internal + local boundary)
    int n_int, n_bnd;                    // scalar unknowns
    int n_own, n_ends, n_slots, n_items;
    SymFactor F;
    std::vector<int> locbus;             // local position -> internal bus id
    std::vector<int> qvarV, qvarT;       // local position -> scalar unknown (-1: none)
    // own buses (internal-numbering order)
    std::vector<int> own_q, own_ebeg, own_sbeg, own_gvv;
    // ends (grouped by own bus, then by neighbour)
    std::vector<int> end_qi, end_qj, end_own, end_var;   // end_var: 4 per end (Vi,Ti,Vj,Tj)
    std::vector<int> end_gpos;           // 10 per end: pairs (a<=b) of (Vi,Ti,Vj,Tj)
    std::vector<int> end_canon;          // canonical row of the P flow row (Q = +L)
    std::vector<double> end_g, end_b, end_bh;
    // neighbour slots of own buses (excluding the bus itself)
    std::vector<int> slot_q, slot_ebeg, slot_ecnt;
    // injection-row gain items: own bus, slot u, slot v (0 = the bus itself), 4 positions
    std::vector<int> item_own, item_uv, item_pos;  // item_uv = u | v << 16
    // packed item records, 4 ints each: {own bus, first end of slot u (-1: the
    // bus itself), first end of slot v, end count u | end count v << 16}
    std::vector<int> item_rec;
    std::vector<int> ebnd;               // local boundary unknown -> boundary-system scalar index
    std::vector<int> bnd_xg;             // local boundary unknown -> x_Gamma index (oracle order)
    long long work = 0;                  // cost estimate for scheduling
    long long g_updates = 0;
};

struct BoundarySetup {
    int n_gamma = 0;                     // scalar unknowns
    int n_bbus = 0;
    SymFactor F;
    std::vector<int> bvar_ibus, bvar_isT;     // boundary scalar -> internal bus id, angle flag
    std::vector<int> xg_of_b;                 // boundary scalar -> x_Gamma index (oracle order)
    std::vector<int> asm_beg;                 // per storage position: gather list range
    std::vector<int> asm_area, asm_off;       // (area, offset within that area's instance storage)
    std::vector<int> rhs_beg, rhs_area, rhs_lv;  // per boundary scalar: (area, local boundary unknown)
};

struct Setup {
    int N = 0, L = 0, K = 0, slack = 0, m = 0;
    std::vector<int> ibus_of_bus, bus_of_ibus;   // canonical <-> internal bus numbering
    std::vector<int> area_of_ibus;
    std::vector<AreaSetup> areas;
    BoundarySetup B;
    std::vector<int> zperm;                      // internal row -> canonical row
    std::vector<int> zrow_base;                  // per area
    int n_boundary_bus = 0;
    std::string error;
};

// Returns false (with s.error set) on invalid input.  An area whose relaxed
// FP32 factor storage would not fit in smem_limit bytes next to its vectors is
// rebuilt with less relaxation (smem_limit 0: no limit).
bool build_setup(const NetIn &net, int n_area, const int32_t *area_of_bus, Setup &s,
                 int smem_limit = kDefaultSmemLimit);

// Host-only consistency check of a setup with random SPD data on its patterns:
// out = {slot-map error, Schur-block error, area solve error, boundary solve error}
// (max relative errors against dense Cholesky).  Returns false with err set if
// a structural inconsistency is found.
bool selfcheck(const Setup &s, unsigned long long seed, double out[4], std::string &err);

}  // namespace mase
