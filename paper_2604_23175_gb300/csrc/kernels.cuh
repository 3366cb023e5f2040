// Device code of libmase (sm_103a).
//
// One thread block works on one (area, snapshot) instance.  The whole local
// pipeline of an iteration (Sec. 4.1-4.3) runs inside it: typed measurement
// templates are evaluated (Eq. typed_meas), the residual, the gradient
// H^T W r (FP64) and the gain matrix G = H^T W H are accumulated straight
// into the area's supernodal factor storage without forming H (Sec. 4.2),
// and the supernodal Cholesky of G_ii with the boundary block ordered last
// leaves the Schur complement S_b and the condensed right-hand side in place
// (Eq. schur_defs, "Schur mode", Sec. 4.3).  The coordinator assembles and
// factors the sparse boundary system per snapshot (Eq. global_assembly,
// Sec. 4.4) and the back-substitution kernel recovers the interior step
// (Eq. backsub).
//
// Precision: RG is the gain/factor/Schur type, RS the type of the local
// triangular solves.  Residuals, the gradient, the boundary refinement and the
// state update are always FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mase_dev {


// Symbolic factor descriptor (all indices relative to its bases).
struct FacDev {
    int n_int, n_bnd, nsn, nlev;
    int store_int, store_total, off_B, max_w;
    int sn_base;       // per-supernode arrays
    int levoff_base;   // lev_off (nlev + 1 entries)
    int rows_base;     // rows / colbase / relbase
    int rel_base;      // rel
    int task_base;     // task_rec (16 ints per task)
    int n_tasks;
    int level_sched;   // 1: tasks grouped by level (lev_tasks), 0: dataflow order
    int levtask_base;  // lev_tasks (3 nlev + 1 entries)
    int chunk_base;    // chunk_rec (8 ints per chunk)
    int levchunk_base; // lev_chunks (nlev + 1 entries)
};

struct AreaDev {
    FacDev F;
    int nb_int, nb_loc, n_own, n_ends, n_slots, n_items;
    int bus_base, own_base, own1_base, end_base, item_base, ebnd_base;
    int zrow_base;
    int in_smem;
    int off_g, off_y, off_bus, off_end, off_inj, off_self, off_st;   // dynamic smem byte offsets
    int smem_bytes;
    int back_smem_bytes;    // dynamic shared memory of the back-substitution (rhs)
    int obj_off_end;        // objective kernel: byte offset of the end flows
    int obj_smem_bytes;     // objective kernel: dynamic shared memory
    // areas whose vectors exceed shared memory (e.g. one area holding the
    // whole network) keep them in global scratch, vec_stride bytes per snapshot
    int vec_global;
    int vec_stride;
    long long vec_base;
    long long fac_base;     // element offset of (area, snapshot 0) in the factor buffer
    int fac_stride;         // elements per snapshot (= store_total)
    long long c_base;       // interior forward-solved rhs, stride n_int
    long long bh_base;      // condensed boundary rhs, stride n_bnd
};

struct Tables {
    const int *sn_c0, *sn_w, *sn_nr, *sn_off, *sn_order;
    const int *lev_off;
    const int *rows, *rel;
    const int *locbus, *qvarV, *qvarT;
    const int *own_q, *own_gvv, *own_ebeg;
    const int *end_qi, *end_qj, *end_own, *end_var, *end_gpos;
    const double *end_g, *end_b, *end_bh;
    const int *item_pos;
    const int *ebnd;
    const int4 *task_rec;   // 4 int4 per factorisation task
    const int *lev_tasks;   // level schedule: group boundaries of the task list
    const int4 *item_rec;   // 1 int4 per injection item
    const int4 *chunk_rec;  // 2 int4 per 32-row panel chunk
    const int *lev_chunks;
    int wait_polls;         // polls of a dataflow wait before it gives up (error bit 4)
    int mma_min_w;          // FP32 factors: update units of panels at least this wide run
                            // on the tensor cores (3xTF32 MMA); 0 = SIMT units only
};

struct StopRule {
    double tol;
    int max_iter;
};

struct State {
    int N, M, S;                 // buses, measurement rows, snapshots
    double *xV, *xT;             // [S][N] internal bus numbering
    const double *z;             // [S][M] internal row order
    const double *W;             // [M] 1/sigma^2
    const uint8_t *mask;         // [S][M] or null
    int *active;                 // [S]
    int *err;                    // [S] bit 1: non-SPD pivot, bit 2: non-finite, bit 4: a bounded wait gave up
    double *J;                   // [S]
    unsigned long long *maxstep; // [S] bit pattern of max |dx| (non-negative double)
    unsigned long long *clk;     // stage clock of this launch: {first block start, last block end}
                                 // in globaltimer ns, or null
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Stage clocks: the first block of a launch to start and the last to finish
// bound the stage's device time (called by thread 0; clk_end after the
// block's last barrier).
__device__ __forceinline__ void clk_begin(unsigned long long *clk) {
    if (clk && threadIdx.x == 0) atomicMin(clk, gtimer());
}
__device__ __forceinline__ void clk_end(unsigned long long *clk) {
    if (clk && threadIdx.x == 0) atomicMax(clk + 1, gtimer());
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t += red[i];
    return t;   // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double *red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
    return t;
}

// P and Q leaving bus i into a branch towards j (pi model, Sec. 2.1 bus-branch
// formulation), from cos/sin of both angles: theta_ij = theta_i - theta_j.
struct EndFlow {
    double P, Q, gc_bs, gs_bc;
};
// g cos(theta_ij) + b sin(theta_ij) and g sin(theta_ij) - b cos(theta_ij) only
__device__ __forceinline__ double2 end_trig(double ci, double si, double cj, double sj, double g,
                                            double b) {
    const double c = ci * cj + si * sj;
    const double s = si * cj - ci * sj;
    return make_double2(g * c + b * s, g * s - b * c);
}
__device__ __forceinline__ EndFlow end_flow(double Vi, double Vj, double ci, double si, double cj,
                                            double sj, double g, double b, double bh) {
    const double c = ci * cj + si * sj;      // cos(theta_i - theta_j)
    const double s = si * cj - ci * sj;      // sin(theta_i - theta_j)
    EndFlow f;
    f.gc_bs = g * c + b * s;
    f.gs_bc = g * s - b * c;
    const double ViVj = Vi * Vj;
    f.P = Vi * Vi * g - ViVj * f.gc_bs;
    f.Q = -Vi * Vi * (b + bh) - ViVj * f.gs_bc;
    return f;
}

// ---------------------------------------------------------------------------
// supernodal factorisation with trailing Schur block + forward solve
// ---------------------------------------------------------------------------

// Factor storage accessors.  Every supernode panel lies wholly in one
// memory, so a panel base is resolved once; update targets are resolved per
// entry.
template <class RG>
struct FlatStore {   // one contiguous block (shared or global memory)
    RG *p;
    __device__ __forceinline__ RG *at(int off) const { return p + off; }
};
template <class RG>
struct SplitStore {  // entries [split, ...) in shared memory, the rest in global memory
    RG *g;
    RG *sm;
    int split;
    __device__ __forceinline__ RG *at(int off) const { return off >= split ? sm + (off - split) : g + off; }
};

template <class RG>
struct ClusterStore {  // entries [split, ...) in cluster block 0's shared memory, the rest in block 1's
    RG *p0;
    RG *p1;
    int split;
    __device__ __forceinline__ RG *at(int off) const { return off >= split ? p0 + (off - split) : p1 + off; }
};

// The threads that run a level-scheduled factorisation or solve: one block,
// or both blocks of a 2-block cluster working on one snapshot.
struct BlockTeam {
    __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ int nwarps() const { return blockDim.x >> 5; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct ClusterTeam {
    int rank;
    __device__ __forceinline__ int warp() const { return rank * (blockDim.x >> 5) + (threadIdx.x >> 5); }
    __device__ __forceinline__ int nwarps() const { return 2 * (blockDim.x >> 5); }
    __device__ __forceinline__ void sync() const {
        // full cluster barrier; orders shared-memory traffic of both blocks
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
};

// Diagonal block of a supernode panel (w <= WB <= 32 columns), by one warp:
// lane r holds row r, column values are broadcast by shuffles; then the
// block's rhs is forward-solved the same way.
template <class RG, class RS, int WB>
__device__ void diag_block(RG *P, int w, int ld, RS *yc, bool do_factor, int lane, int *err) {
    constexpr unsigned FULL = 0xffffffffu;
    RG a[WB];
#pragma unroll
    for (int c = 0; c < WB; ++c)
        a[c] = (c < w && lane < w && c <= lane) ? P[(size_t)c * ld + lane] : RG(0);
    if (do_factor) {
#pragma unroll
        for (int c = 0; c < WB; ++c) {
            if (c < w) {
                RG d = __shfl_sync(FULL, a[c], c);
                if (!(d > RG(0))) {
                    if (lane == 0) atomicOr(err, 1);
                    d = RG(1);
                }
                // the diagonal entry is stored as its reciprocal 1/L_cc so that
                // every later solve multiplies instead of dividing
                const RG inv = rsqrt(d);
                if (lane == c) a[c] = inv;
                else if (lane > c) a[c] *= inv;
                // branch-free so the independent shuffles pipeline; columns >= w
                // only ever touch entries outside the block
#pragma unroll
                for (int c2 = c + 1; c2 < WB; ++c2) {
                    const RG l = __shfl_sync(FULL, a[c], c2);   // L[c2][c]
                    a[c2] = lane >= c2 ? a[c2] - a[c] * l : a[c2];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < WB; ++c)
            if (c < w && lane < w && c <= lane) P[(size_t)c * ld + lane] = a[c];
    }
    RS yl = lane < w ? yc[lane] : RS(0);
#pragma unroll
    for (int c = 0; c < WB; ++c) {
        if (c < w) {
            const RS yv = __shfl_sync(FULL, yl, c) * RS(__shfl_sync(FULL, a[c], c));
            if (lane == c) yl = yv;
            else if (lane > c && lane < w) yl -= RS(a[c]) * yv;
        }
    }
    if (lane < w) yc[lane] = yl;
}

// Rows r0 .. r0+32 of a panel below its factored diagonal block, by one warp
// (lane = row): forward substitution against the block, right-looking so the
// multiply-adds are independent, L read from shared memory.
template <class RG, int WB>
__device__ void panel_rows(RG *P, int w, int ld, int r0, int lane) {
    const int row = r0 + lane;
    if (row >= ld) return;
    RG x[WB];
#pragma unroll
    for (int c = 0; c < WB; ++c) x[c] = c < w ? P[(size_t)c * ld + row] : RG(0);
    // branch-free inner loop; loads beyond column w are replaced by zero
#pragma unroll
    for (int c = 0; c < WB; ++c) {
        if (c < w) {
            const RG *Lc = P + (size_t)c * ld;
            x[c] *= Lc[c];
#pragma unroll
            for (int c2 = c + 1; c2 < WB; ++c2) {
                const RG l = c2 < w ? Lc[c2] : RG(0);
                x[c2] -= x[c] * l;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < WB; ++c)
        if (c < w) P[(size_t)c * ld + row] = x[c];
}

// Diagonal block wider than 16 columns as a 2 x 2 block Cholesky: factor the
// leading 16 columns, solve the rows 16..w-1 against them, update the trailing
// block and its rhs, factor the trailing block.  No step holds more than 16
// values per lane, so the tile stays in registers.
template <class RG, class RS>
__device__ void diag_block_wide(RG *P, int w, int ld, RS *yc, bool do_factor, int lane, int *err) {
    constexpr int H = 16;
    diag_block<RG, RS, H>(P, H, ld, yc, do_factor, lane, err);
    __syncwarp();
    const int r = H + lane;
    const bool mine = lane < w - H;
    if (do_factor) {
        // L21 = A21 L11^-T for the rows H..w-1 of the block
        RG x[H];
#pragma unroll
        for (int c = 0; c < H; ++c) x[c] = mine ? P[(size_t)c * ld + r] : RG(0);
#pragma unroll
        for (int c = 0; c < H; ++c) {
            const RG *Lc = P + (size_t)c * ld;
            x[c] *= Lc[c];
#pragma unroll
            for (int c2 = c + 1; c2 < H; ++c2) x[c2] -= x[c] * Lc[c2];
        }
        if (mine) {
#pragma unroll
            for (int c = 0; c < H; ++c) P[(size_t)c * ld + r] = x[c];
        }
        __syncwarp();
        // A22 -= L21 L21^T (lower part): lane r updates its row
        if (mine) {
            for (int c2 = H; c2 <= r; ++c2) {
                RG v = RG(0);
#pragma unroll
                for (int k = 0; k < H; ++k) v += x[k] * P[(size_t)k * ld + c2];
                P[(size_t)c2 * ld + r] -= v;
            }
        }
    }
    // rhs of the trailing rows: y2 -= L21 y1
    if (mine) {
        RS v = RS(0);
#pragma unroll
        for (int k = 0; k < H; ++k) v += RS(P[(size_t)k * ld + r]) * yc[k];
        yc[r] -= v;
    }
    __syncwarp();
    diag_block<RG, RS, H>(P + (size_t)H * ld + H, w - H, ld, yc + H, do_factor, lane, err);
}

template <class RG, class RS>
__device__ __forceinline__ void diag_block_any(RG *P, int w, int ld, RS *yc, bool do_factor,
                                               int lane, int *err) {
    if (w <= 2) diag_block<RG, RS, 2>(P, w, ld, yc, do_factor, lane, err);
    else if (w <= 4) diag_block<RG, RS, 4>(P, w, ld, yc, do_factor, lane, err);
    else if (w <= 8) diag_block<RG, RS, 8>(P, w, ld, yc, do_factor, lane, err);
    else if (w <= 16) diag_block<RG, RS, 16>(P, w, ld, yc, do_factor, lane, err);
    else diag_block_wide<RG, RS>(P, w, ld, yc, do_factor, lane, err);
}

// ---------------------------------------------------------------------------
// Register-staged variants for a factor spread over both blocks of a cluster.
// There half of every panel lies in the other block's shared memory, whose
// loads take hundreds of cycles; the substitution chains above would wait on
// one such load per column.  Here each lane first loads its own row (or
// column) of the block in one go, and the chains move values between lanes
// with shuffles only.
// ---------------------------------------------------------------------------
// (FP32 factors only: an FP64 block of 32 x 32 does not fit the registers.)
template <class ST>
struct RemoteStore {
    static constexpr bool value = false;
};
template <>
struct RemoteStore<ClusterStore<float>> {
    static constexpr bool value = true;
};

// panel_rows with the factored diagonal block held by rows in the lanes
// (lane k: row k; 1/L_kk on its diagonal).  All lanes take part in the
// shuffles; rows past the panel are computed on zeros and not stored.
template <class RG, int WB>
__device__ void panel_rows_reg(RG *P, int w, int ld, int r0, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    const int row = r0 + lane;
    const bool mine = row < ld;
    RG Lr[WB], x[WB];
#pragma unroll
    for (int c = 0; c < WB; ++c) {
        Lr[c] = (c < w && lane < w && c <= lane) ? P[(size_t)c * ld + lane] : RG(0);
        x[c] = (mine && c < w) ? P[(size_t)c * ld + row] : RG(0);
    }
#pragma unroll
    for (int c = 0; c < WB; ++c) {
        if (c < w) {
            x[c] *= __shfl_sync(FULL, Lr[c], c);
#pragma unroll
            for (int c2 = c + 1; c2 < WB; ++c2) x[c2] -= x[c] * __shfl_sync(FULL, Lr[c], c2);
        }
    }
    if (mine) {
#pragma unroll
        for (int c = 0; c < WB; ++c)
            if (c < w) P[(size_t)c * ld + row] = x[c];
    }
}

template <class RG>
__device__ __forceinline__ void panel_rows_reg_any(RG *P, int w, int ld, int r0, int lane) {
    if (w <= 8) panel_rows_reg<RG, 8>(P, w, ld, r0, lane);
    else if (w <= 16) panel_rows_reg<RG, 16>(P, w, ld, r0, lane);
    else panel_rows_reg<RG, 32>(P, w, ld, r0, lane);
}

// diag_block_wide with the solve of the rows H..w-1 against L11 and the
// trailing update done on registers: L11's rows are reloaded by the lanes
// that hold them, L21's rows stay in the lanes that computed them.
template <class RG, class RS>
__device__ void diag_block_wide_reg(RG *P, int w, int ld, RS *yc, int lane, int *err) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int H = 16;
    diag_block<RG, RS, H>(P, H, ld, yc, true, lane, err);
    __syncwarp();
    const int r = H + lane;
    const bool mine = lane < w - H;
    RG Lr[H], x[H];
#pragma unroll
    for (int c = 0; c < H; ++c) {
        Lr[c] = (lane < H && c <= lane) ? P[(size_t)c * ld + lane] : RG(0);
        x[c] = mine ? P[(size_t)c * ld + r] : RG(0);
    }
    // L21 = A21 L11^-T
#pragma unroll
    for (int c = 0; c < H; ++c) {
        x[c] *= __shfl_sync(FULL, Lr[c], c);
#pragma unroll
        for (int c2 = c + 1; c2 < H; ++c2) x[c2] -= x[c] * __shfl_sync(FULL, Lr[c], c2);
    }
    if (mine) {
#pragma unroll
        for (int c = 0; c < H; ++c) P[(size_t)c * ld + r] = x[c];
    }
    // A22 -= L21 L21^T (lower part): row H + j of L21 is lane j's x
#pragma unroll
    for (int j = 0; j < H; ++j) {
        if (j < w - H) {
            RG v = RG(0);
#pragma unroll
            for (int k = 0; k < H; ++k) v += x[k] * __shfl_sync(FULL, x[k], j);
            if (mine && j <= lane) P[(size_t)(H + j) * ld + r] -= v;
        }
    }
    // rhs of the trailing rows: y2 -= L21 y1
    if (mine) {
        RS v = RS(0);
#pragma unroll
        for (int k = 0; k < H; ++k) v += RS(x[k]) * yc[k];
        yc[r] -= v;
    }
    __syncwarp();
    diag_block<RG, RS, H>(P + (size_t)H * ld + H, w - H, ld, yc + H, true, lane, err);
}

template <class RG>
__device__ __forceinline__ void panel_rows_any(RG *P, int w, int ld, int r0, int lane) {
    if (w <= 2) panel_rows<RG, 2>(P, w, ld, r0, lane);
    else if (w <= 4) panel_rows<RG, 4>(P, w, ld, r0, lane);
    else if (w <= 8) panel_rows<RG, 8>(P, w, ld, r0, lane);
    else if (w <= 16) panel_rows<RG, 16>(P, w, ld, r0, lane);
    else panel_rows<RG, 32>(P, w, ld, r0, lane);
}

// Updates of one unit: NJ target columns j0 .. j0+NJ of a supernode's row set,
// for the rows i >= j0.  A pass covers MC 32-row chunks (lane = row within a
// chunk), so every target-column value loaded from shared memory serves MC
// rows; rows i < rhs_end also update the rhs (the unit that starts a target
// segment carries that segment's rows).  Index loads are issued up front.
template <class RG, class RS, int NJ, int MC, class ST>
__device__ __forceinline__ void unit_pass(const ST &st, RS *y, const RG *Ps, const int *relp,
                                          const int *rws, const RS *yc, int w, int ld, int j0,
                                          int rhs_end, const int (&cb)[4], int i0, int lane) {
    const int R = ld - w;
    int ir[MC], tg[MC], rw[MC];
    bool ok[MC], rh[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        ir[m] = i0 + 32 * m + lane;
        ok[m] = ir[m] < R;
        rh[m] = ir[m] < rhs_end;
        tg[m] = ok[m] ? relp[ir[m]] : 0;
        rw[m] = rh[m] ? rws[ir[m]] : 0;
    }
    const bool any_rhs = i0 < rhs_end;
    RG v[MC][NJ];
    RS vr[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        vr[m] = RS(0);
#pragma unroll
        for (int k = 0; k < NJ; ++k) v[m][k] = RG(0);
    }
    for (int c = 0; c < w; ++c) {
        const RG *col = Ps + (size_t)c * ld;
        RG lj[NJ];
#pragma unroll
        for (int k = 0; k < NJ; ++k) lj[k] = col[j0 + k];
        const RS ycc = any_rhs ? yc[c] : RS(0);
#pragma unroll
        for (int m = 0; m < MC; ++m) {
            const RG li = ok[m] ? col[ir[m]] : RG(0);
#pragma unroll
            for (int k = 0; k < NJ; ++k) v[m][k] += li * lj[k];
            vr[m] += RS(li) * ycc;
        }
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        if (ok[m]) {
#pragma unroll
            for (int k = 0; k < NJ; ++k)
                if (ir[m] >= j0 + k) atomicAdd(st.at(cb[k] + tg[m]), -v[m][k]);
        }
        if (rh[m]) atomicAdd(y + rw[m], -vr[m]);
    }
}

template <class RG, class RS, int NJ, class ST>
__device__ __forceinline__ void unit_rows(const ST &st, RS *y, const RG *Ps, const int *relp,
                                          const int *rws, const RS *yc, int w, int ld, int j0,
                                          int rhs_end, const int (&cb)[4], int lane) {
    const int R = ld - w;
    int i0 = j0;
    for (; i0 + 64 < R; i0 += 96)
        unit_pass<RG, RS, NJ, 3, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, i0, lane);
    if (i0 + 32 < R)
        unit_pass<RG, RS, NJ, 2, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, i0, lane);
    else if (i0 < R)
        unit_pass<RG, RS, NJ, 1, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, i0, lane);
}

// Update unit on the tensor cores (FP32 factors only): the same products as
// unit_rows, as warp-level m16n8k8 TF32 MMAs.  A is the unit's rows of the
// panel (16 rows per tile, the panel's columns as k), B holds the unit's
// target columns (n = 0..nj-1) and, in n = 4, the supernode's rhs values, so
// that the rhs update rides along.  Each operand is split into a TF32 high
// part and a TF32 remainder, and hi*hi + hi*lo + lo*hi are accumulated in
// FP32 ("3xTF32"), which keeps the products at FP32 accuracy (a single TF32
// product would carry a 2^-11 relative error into the Gauss-Newton step).
// Results are scattered like unit_rows's: the lane holding (row, n) adds it
// to the target through the relative-index map (n < nj, lower triangle) or
// to the rhs row (n = 4, rows below rhs_end).
__device__ __forceinline__ unsigned tf32_hi(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <int KS, class ST>
__device__ __forceinline__ void unit_mma(const ST &st, float *y, const float *Ps, const int *relp,
                                         const int *rws, const float *yc, int w, int ld, int j0,
                                         int nj, int rhs_end, const int (&cb)[4], int lane) {
    const int R = ld - w;
    const int g = lane >> 2, t = lane & 3;
    // B fragments: b0 = B[k = t][n = g], b1 = B[k = t + 4][n = g] of each k-step
    unsigned bh[KS][2], bl[KS][2];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 8 * ks + t + 4 * h;
            float b = 0.f;
            if (k < w) {
                if (g < nj) b = Ps[(size_t)k * ld + j0 + g];
                else if (g == 4 && rhs_end > 0) b = yc[k];
            }
            bh[ks][h] = tf32_hi(b);
            bl[ks][h] = tf32_hi(b - __uint_as_float(bh[ks][h]));
        }
    for (int r0 = j0; r0 < R; r0 += 16) {
        const int ra = r0 + g, rb = r0 + g + 8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            // a0 = A[g][t], a1 = A[g + 8][t], a2 = A[g][t + 4], a3 = A[g + 8][t + 4]
            const int k0 = 8 * ks + t, k1 = k0 + 4;
            const float x0 = (ra < R && k0 < w) ? Ps[(size_t)k0 * ld + ra] : 0.f;
            const float x1 = (rb < R && k0 < w) ? Ps[(size_t)k0 * ld + rb] : 0.f;
            const float x2 = (ra < R && k1 < w) ? Ps[(size_t)k1 * ld + ra] : 0.f;
            const float x3 = (rb < R && k1 < w) ? Ps[(size_t)k1 * ld + rb] : 0.f;
            const unsigned ah[4] = {tf32_hi(x0), tf32_hi(x1), tf32_hi(x2), tf32_hi(x3)};
            const unsigned al[4] = {tf32_hi(x0 - __uint_as_float(ah[0])), tf32_hi(x1 - __uint_as_float(ah[1])),
                                    tf32_hi(x2 - __uint_as_float(ah[2])), tf32_hi(x3 - __uint_as_float(ah[3]))};
            mma_tf32(acc, al, bh[ks][0], bh[ks][1]);
            mma_tf32(acc, ah, bl[ks][0], bl[ks][1]);
            mma_tf32(acc, ah, bh[ks][0], bh[ks][1]);
        }
        // c0 = C[g][2t], c1 = C[g][2t + 1], c2 = C[g + 8][2t], c3 = C[g + 8][2t + 1]
        if (t < 2) {
            const int n0 = 2 * t, n1 = n0 + 1;
            if (ra < R) {
                const int tr = relp[ra];
                if (n0 < nj && ra >= j0 + n0) atomicAdd(st.at(cb[n0] + tr), -acc[0]);
                if (n1 < nj && ra >= j0 + n1) atomicAdd(st.at(cb[n1] + tr), -acc[1]);
            }
            if (rb < R) {
                const int tr = relp[rb];
                if (n0 < nj && rb >= j0 + n0) atomicAdd(st.at(cb[n0] + tr), -acc[2]);
                if (n1 < nj && rb >= j0 + n1) atomicAdd(st.at(cb[n1] + tr), -acc[3]);
            }
        } else if (t == 2) {
            if (ra < rhs_end) atomicAdd(y + rws[ra], -acc[0]);
            if (rb < rhs_end) atomicAdd(y + rws[rb], -acc[2]);
        }
    }
}

// Task bodies are kept out of line so that each gets the whole register file
// for its own tile (a diagonal tile of up to 16 columns lives in 16 registers
// per lane) and no tile spills.
template <class RG, class RS, class ST>
__device__ __noinline__ void task_diag(const ST st, int off, int w, int ld, RS *yc, int *err) {
    if constexpr (RemoteStore<ST>::value) {
        if (w > 16 && w <= 32) {
            diag_block_wide_reg<RG, RS>(st.at(off), w, ld, yc, threadIdx.x & 31, err);
            return;
        }
    }
    diag_block_any<RG, RS>(st.at(off), w, ld, yc, true, threadIdx.x & 31, err);
}
template <class RG, class ST>
__device__ __noinline__ void task_panel(const ST st, int off, int w, int ld, int r0) {
    if constexpr (RemoteStore<ST>::value) {
        if (w <= 32) {
            panel_rows_reg_any<RG>(st.at(off), w, ld, r0, threadIdx.x & 31);
            return;
        }
    }
    panel_rows_any<RG>(st.at(off), w, ld, r0, threadIdx.x & 31);
}
template <class RG, class RS, class ST>
__device__ __noinline__ void task_unit(const ST st, RS *y, const int *rel, const int *rows,
                                       const int4 q1, const int4 q2, const int4 q3, int mma_min_w) {
    const int lane = threadIdx.x & 31;
    const RG *Ps = st.at(q1.x);
    const int *relp = rel + q1.y;
    const int *rws = rows + q1.z;
    const RS *yc = y + q1.w;
    const int w = q2.x & 0xff, nj = q2.x >> 8, ld = q2.y & 0xffff, j0 = q2.y >> 16;
    const int rhs_end = q2.z;
    const int cb[4] = {q2.w, q3.x, q3.y, q3.z};
    if constexpr (std::is_same<RG, float>::value && std::is_same<RS, float>::value) {
        if (mma_min_w > 0 && w >= mma_min_w) {
            if (w <= 8) unit_mma<1, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, nj, rhs_end, cb, lane);
            else if (w <= 16) unit_mma<2, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, nj, rhs_end, cb, lane);
            else unit_mma<4, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, nj, rhs_end, cb, lane);
            return;
        }
    }
    switch (nj) {
        case 1: unit_rows<RG, RS, 1, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, lane); break;
        case 2: unit_rows<RG, RS, 2, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, lane); break;
        case 3: unit_rows<RG, RS, 3, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, lane); break;
        default: unit_rows<RG, RS, 4, ST>(st, y, Ps, relp, rws, yc, w, ld, j0, rhs_end, cb, lane); break;
    }
}

// Numeric factorisation + forward solve as a dataflow over the task list
// (diagonal blocks, panel chunks, update units).  A free warp takes the next
// task index from a shared counter, waits (bounded) until the task's counter
// reaches its threshold, runs it and signals its own counter.  Tasks are in a
// topological order, so the lowest unfinished task can always run.  Updates
// of ancestors, of the trailing Schur block and of the rhs are scattered with
// shared/global atomics through the relative-index maps.  ctr holds 2 nsn + 1
// ints of shared memory.  Must be called by every thread of the block.
template <class RG, class RS, class ST>
__device__ void factor_tasks(const FacDev &F, const Tables &T, const ST &st, RS *y, int *ctr,
                             int *err) {
    constexpr unsigned FULL = 0xffffffffu;
    const int wait_limit = T.wait_polls;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int nsn = F.nsn, ntask = F.n_tasks;
    for (int i = tid; i <= 2 * nsn; i += nt) ctr[i] = 0;
    __syncthreads();
    const int4 *trec = T.task_rec + 4 * (long long)F.task_base;
    const int *rel = T.rel + F.rel_base;
    const int *rows = T.rows + F.rows_base;
    int *next = ctr + 2 * nsn;
    for (;;) {
        // a warp takes the next task only when it is free, so a task on the
        // critical path never queues behind a long one
        int t = 0;
        if (lane == 0) t = atomicAdd(next, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        // the record a warp will take about one round of grabs later, into L1
        if (lane == 0 && t + 16 < ntask)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(trec + 4 * (t + 16)));
        const int4 q0 = trec[4 * t], q1 = trec[4 * t + 1], q2 = trec[4 * t + 2], q3 = trec[4 * t + 3];
        if (lane == 0 && q0.z > 0) {
            const volatile int *c = ctr + q0.y;
            int it = 0;
            while (*c < q0.z) {
                if (++it >= wait_limit) {
                    atomicOr(err, 4);
                    break;
                }
                __nanosleep(32);
            }
            __threadfence_block();
        }
        __syncwarp();
        const int type = q0.x >> 24;
        if (type == 0) task_diag<RG, RS, ST>(st, q1.x, q1.y, q1.z, y + q1.w, err);
        else if (type == 1) task_panel<RG, ST>(st, q1.x, q1.y, q1.z, q1.w);
        else task_unit<RG, RS, ST>(st, y, rel, rows, q1, q2, q3, T.mma_min_w);
        __syncwarp();
        if (lane == 0 && q0.w >= 0) {
            __threadfence_block();
            atomicAdd(ctr + q0.w, 1);
        }
    }
    __syncthreads();
}

// The same factorisation with a level schedule: per level, the diagonal
// blocks, then the panel chunks, then the update units, each group spread over
// the warps and closed by a block barrier.  Suits factors whose top levels are
// wide (the boundary system) better than the dataflow.
template <class RG, class RS, class ST, class TM = BlockTeam>
__device__ void factor_levels(const FacDev &F, const Tables &T, const ST &st, RS *y, int *err,
                              const TM &tm = TM()) {
    const int warp = tm.warp(), nw = tm.nwarps();
    const int4 *trec = T.task_rec + 4 * (long long)F.task_base;
    const int *lt = T.lev_tasks + F.levtask_base;
    const int *rel = T.rel + F.rel_base;
    const int *rows = T.rows + F.rows_base;
    for (int g = 0; g < 3 * F.nlev; ++g) {
        const int a = lt[g], e = lt[g + 1];
        if (a == e) continue;
        for (int t = a + warp; t < e; t += nw) {
            const int4 q1 = trec[4 * t + 1];
            const int type = g % 3;
            if (type == 0) {
                task_diag<RG, RS, ST>(st, q1.x, q1.y, q1.z, y + q1.w, err);
            } else if (type == 1) {
                task_panel<RG, ST>(st, q1.x, q1.y, q1.z, q1.w);
            } else {
                const int4 q2 = trec[4 * t + 2], q3 = trec[4 * t + 3];
                task_unit<RG, RS, ST>(st, y, rel, rows, q1, q2, q3, T.mma_min_w);
            }
        }
        tm.sync();
    }
}

template <class RG, class RS, class ST>
__device__ __forceinline__ void factor_numeric(const FacDev &F, const Tables &T, const ST &st, RS *y,
                                               int *ctr, int *err) {
    if (F.level_sched) factor_levels<RG, RS, ST>(F, T, st, y, err);
    else factor_tasks<RG, RS, ST>(F, T, st, y, ctr, err);
}

// Forward solve L y = b with a factored storage, level by level: diagonal
// blocks by one warp each, then the rhs updates of the rows below them in
// 32-row chunks over all warps.  Must be called by every thread of the block.
template <class RG, class RS, class ST, class TM = BlockTeam>
__device__ void solve_forward(const FacDev &F, const Tables &T, const ST &st, RS *y,
                              const TM &tm = TM()) {
    const int lane = threadIdx.x & 31, warp = tm.warp(), nw = tm.nwarps();
    const int *sn_order = T.sn_order + F.sn_base;
    const int *lev_off = T.lev_off + F.levoff_base;
    const int *lev_chunks = T.lev_chunks + F.levchunk_base;
    const int4 *crec = T.chunk_rec + 2 * (long long)F.chunk_base;
    const int *rows = T.rows + F.rows_base;
    for (int lev = 0; lev < F.nlev; ++lev) {
        const int a = lev_off[lev], e = lev_off[lev + 1];
        for (int i = a + warp; i < e; i += nw) {
            const int s = F.sn_base + sn_order[i];
            const int w = T.sn_w[s];
            diag_block_any<RG, RS>(st.at(T.sn_off[s]), w, w + T.sn_nr[s], y + T.sn_c0[s], false,
                                   lane, nullptr);
        }
        tm.sync();
        for (int k = lev_chunks[lev] + warp; k < lev_chunks[lev + 1]; k += nw) {
            const int4 r = crec[2 * k], r2 = crec[2 * k + 1];
            const RG *P = st.at(r.x);
            const int w = r.y, ld = r.z, row = r.w + lane;
            if (row < ld) {
                const RS *yc = y + r2.x;
                RS v = RS(0);
                for (int c = 0; c < w; ++c) v += RS(P[(size_t)c * ld + row]) * yc[c];
                atomicAdd(y + rows[r2.y + row - w], -v);
            }
        }
        tm.sync();
    }
}

// Column sums sum_rows P[c][row] * xi of one 32-row chunk of a panel (lane =
// row, w <= WB columns): a transpose-reduction of the lanes' WB products (the
// lanes exchange halves of their columns at distances WB/2 .. 1, WB - 1
// exchanges in all, after folding the two half-warps when WB = 16).  Lane c
// returns column c.
template <class RG, class RS, int WB>
__device__ __forceinline__ RS chunk_colsum(const RG *P, int w, int ld, int row, RS xi, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    const bool ok = row < ld;
    RS v[WB];
#pragma unroll
    for (int c = 0; c < WB; ++c) v[c] = (ok && c < w) ? RS(P[(size_t)c * ld + row]) * xi : RS(0);
    if (WB == 16) {
#pragma unroll
        for (int c = 0; c < WB; ++c) v[c] += __shfl_xor_sync(FULL, v[c], 16);
    }
#pragma unroll
    for (int d = WB / 2; d >= 1; d >>= 1) {
        const bool up = (lane & d) != 0;
#pragma unroll
        for (int k = 0; k < d; ++k) {
            const RS send = up ? v[k] : v[k + d];
            const RS keep = up ? v[k + d] : v[k];
            v[k] = keep + __shfl_xor_sync(FULL, send, d);
        }
    }
    return v[0];
}

// Backward substitution with one diagonal block of at most 32 columns on
// registers (lane r loads column r of L; 1/L_cc on the diagonal).
template <class RG, class RS>
__device__ __forceinline__ void back_diag_reg(const RG *P, int w, int ld, RS *yc, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    RG col[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) col[c] = (lane < w && c >= lane && c < w) ? P[(size_t)lane * ld + c] : RG(0);
    RS t = lane < w ? yc[lane] : RS(0);
#pragma unroll
    for (int c = 31; c >= 0; --c) {
        if (c < w) {
            const RS xc = __shfl_sync(FULL, t * RS(col[c]), c);
            if (lane == c) t = xc;
            else if (lane < c) t -= RS(col[c]) * xc;
        }
    }
    if (lane < w) yc[lane] = t;
}

// Backward solve L^T x = y over the internal supernodes, top level first.
// y[n_int..] must hold the (already known) boundary unknowns; on return
// y[0..n_int) holds the interior solution (Eq. backsub).
template <class RG, class RS, class ST, class TM = BlockTeam>
__device__ void back_solve(const FacDev &F, const Tables &T, const ST &st, RS *y,
                           const TM &tm = TM()) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = tm.warp(), nw = tm.nwarps();
    const int *sn_order = T.sn_order + F.sn_base;
    const int *lev_off = T.lev_off + F.levoff_base;
    const int *lev_chunks = T.lev_chunks + F.levchunk_base;
    const int4 *crec = T.chunk_rec + 2 * (long long)F.chunk_base;
    const int *rows = T.rows + F.rows_base;
    for (int lev = F.nlev - 1; lev >= 0; --lev) {
        // (a) contributions of the (already solved) rows below each diagonal block,
        //     32-row chunks over all warps, reduced per column
        for (int k = lev_chunks[lev] + warp; k < lev_chunks[lev + 1]; k += nw) {
            const int4 r = crec[2 * k], r2 = crec[2 * k + 1];
            const RG *P = st.at(r.x);
            const int w = r.y, ld = r.z, row = r.w + lane;
            const RS xi = row < ld ? y[rows[r2.y + row - w]] : RS(0);
            RS sum;
            if (w <= 16) sum = chunk_colsum<RG, RS, 16>(P, w, ld, row, xi, lane);
            else sum = chunk_colsum<RG, RS, 32>(P, w, ld, row, xi, lane);
            if (lane < w) atomicAdd(y + r2.x + lane, -sum);
        }
        tm.sync();
        // (b) backward substitution with the diagonal block (lane r holds y_r)
        const int a = lev_off[lev], e = lev_off[lev + 1];
        for (int i = a + warp; i < e; i += nw) {
            const int s = F.sn_base + sn_order[i];
            const int w = T.sn_w[s], ld = w + T.sn_nr[s], c0 = T.sn_c0[s];
            const RG *P = st.at(T.sn_off[s]);
            if constexpr (RemoteStore<ST>::value) {
                if (w <= 32) {
                    back_diag_reg<RG, RS>(P, w, ld, y + c0, lane);
                    continue;
                }
            }
            for (int kb = ((w - 1) / 32) * 32; kb >= 0; kb -= 32) {
                const int r = kb + lane;
                RS t = r < w ? y[c0 + r] : RS(0);
                for (int c = min(w, kb + 32) - 1; c >= kb; --c) {
                    const RS xc = __shfl_sync(FULL, t * RS(P[(size_t)c * ld + c]), c - kb);
                    if (lane == c - kb) t = xc;
                    else if (r < c) t -= RS(P[(size_t)r * ld + c]) * xc;
                }
                if (r < w) y[c0 + r] = t;
                __syncwarp();
                // earlier column blocks of a panel wider than 32 see this block's solution
                for (int rr = lane; rr < kb; rr += 32) {
                    RS v = RS(0);
                    for (int c = kb; c < min(w, kb + 32); ++c) v += RS(P[(size_t)rr * ld + c]) * y[c0 + c];
                    y[c0 + rr] -= v;
                }
                __syncwarp();
            }
        }
        tm.sync();
    }
}

// ---------------------------------------------------------------------------
// local kernel: evaluation + fused accumulation + Schur condensation
// ---------------------------------------------------------------------------
// VG: some areas keep their vectors in global scratch (vscratch); compiled
// separately so that the usual all-on-chip kernel addresses shared memory only.
template <class RG, class RS, bool VG>
__global__ void __launch_bounds__(512) k_local(const AreaDev *__restrict__ areas, Tables T, State X,
                                               const int2 *__restrict__ inst, int area_only,
                                               RG *fac, RS *cvec, double *bh, unsigned char *vscratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_err;
    int k, s;
    if (area_only >= 0) {
        k = area_only;
        s = blockIdx.x;
    } else {
        const int2 ks = inst[blockIdx.x];
        k = ks.x;
        s = ks.y;
    }
    if (!X.active[s]) return;
    clk_begin(X.clk);
    const AreaDev A = areas[k];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nv = A.F.n_int + A.F.n_bnd;
    const bool vglob = VG && A.vec_global;
    unsigned char *vb = vglob ? vscratch + A.vec_base + (long long)s * A.vec_stride : smem;
    double *g = (double *)(vb + A.off_g);
    RS *y = (RS *)(vb + A.off_y);
    double *bV = (double *)(vb + A.off_bus);
    double *bC = bV + A.nb_loc;
    double *bS = bC + A.nb_loc;
    unsigned char *endbuf = vb + A.off_end;
    double2 *inj = (double2 *)(vb + A.off_inj);
    RG *self = (RG *)(vb + A.off_self);
    RG *st = A.in_smem ? (RG *)(vb + A.off_st) : fac + A.fac_base + (long long)s * A.fac_stride;
    // dataflow counters: the bus-value region once evaluation is done, or the
    // block's own shared memory when the vectors are global
    int *ctr = vglob ? (int *)smem : (int *)(vb + A.off_bus);
    const int endstride = (4 * sizeof(RG) > 16) ? 4 * (int)sizeof(RG) : 16;

    const long long zb = (long long)s * X.M + A.zrow_base;
    const double *z = X.z + zb;
    const double *Wr = X.W + A.zrow_base;
    const uint8_t *mk = X.mask ? X.mask + zb : nullptr;
    auto wt = [&](int r) { return mk ? (mk[r] ? Wr[r] : 0.0) : Wr[r]; };
    const int n_own = A.n_own, n_ends = A.n_ends;
    const int rV = 0, rP = n_own, rQ = 2 * n_own, rPe = 3 * n_own, rQe = 3 * n_own + n_ends;

    if (tid == 0) s_err = 0;
    // ---- E0: bus values, zero accumulators
    for (int q = tid; q < A.nb_loc; q += nt) {
        const int ib = T.locbus[A.bus_base + q];
        const double V = X.xV[(long long)s * X.N + ib], th = X.xT[(long long)s * X.N + ib];
        double sn, cs;
        sincos(th, &sn, &cs);
        bV[q] = V;
        bC[q] = cs;
        bS[q] = sn;
    }
    for (int i = tid; i < nv; i += nt) g[i] = 0.0;
    for (int i = tid; i < A.F.store_total; i += nt) st[i] = RG(0);
    for (int i = tid; i < 4 * n_own; i += nt) self[i] = RG(0);
    __syncthreads();
    // ---- E1: flows at every owned branch end (FP64)
    for (int e = tid; e < n_ends; e += nt) {
        const int ee = A.end_base + e;
        const int qi = T.end_qi[ee], qj = T.end_qj[ee];
        const EndFlow f = end_flow(bV[qi], bV[qj], bC[qi], bS[qi], bC[qj], bS[qj], T.end_g[ee],
                                   T.end_b[ee], T.end_bh[ee]);
        double2 *pq = (double2 *)(endbuf + (size_t)e * endstride);
        *pq = make_double2(f.P, f.Q);
    }
    __syncthreads();
    // ---- E2: voltage rows and injection residuals per own bus
    double Jloc = 0.0;
    for (int o = tid; o < n_own; o += nt) {
        const int q = T.own_q[A.own_base + o];
        const double V = bV[q];
        const double wv = wt(rV + o), rv = z[rV + o] - V;
        Jloc += wv * rv * rv;
        double Pi = 0.0, Qi = 0.0;
        const int e0 = T.own_ebeg[A.own1_base + o], e1 = T.own_ebeg[A.own1_base + o + 1];
        for (int e = e0; e < e1; ++e) {
            const double2 pq = *(const double2 *)(endbuf + (size_t)e * endstride);
            Pi += pq.x;
            Qi += pq.y;
        }
        const double wp = wt(rP + o), wq = wt(rQ + o);
        const double rp = z[rP + o] - Pi, rq = z[rQ + o] - Qi;
        Jloc += wp * rp * rp + wq * rq * rq;
        inj[o] = make_double2(wp * rp, wq * rq);
        atomicAdd(g + T.qvarV[A.bus_base + q], wv * rv);
        atomicAdd(st + T.own_gvv[A.own_base + o], RG(wv));
    }
    __syncthreads();
    // ---- E3: flow rows; gradient of flow and injection rows; flow-row gain terms.
    // Ends are grouped by owning bus, so the lanes of a warp hold runs of ends
    // of one bus: the terms every end of a bus adds to the same place (the
    // bus's own gradient entries and diagonal gain block, its injection self
    // partials) are summed over each run by a warp-level segmented reduction
    // and added once per run; the terms aimed at the far bus are added per end.
    {
        constexpr unsigned FULL = 0xffffffffu;
        const int lane = tid & 31;
        for (int e0 = tid - lane; e0 < n_ends; e0 += nt) {
            const int e = e0 + lane;
            const bool valid = e < n_ends;
            const int ee = A.end_base + (valid ? e : 0);
            double own_g[2] = {0.0, 0.0};   // gradient of the own bus's V and theta
            RG own_s[7];                     // gain (Vi,Vi), (Vi,thi), (thi,thi); self partials
#pragma unroll
            for (int q = 0; q < 7; ++q) own_s[q] = RG(0);
            int o = -1 - lane, gv0 = -1, gv1 = -1, gp0 = -1, gp1 = -1, gp4 = -1;
            if (valid) {
                const int qi = T.end_qi[ee], qj = T.end_qj[ee];
                const double2 pq = *(const double2 *)(endbuf + (size_t)e * endstride);
                const double wPe = wt(rPe + e), wQe = wt(rQe + e);
                const double rPf = z[rPe + e] - pq.x, rQf = z[rQe + e] - pq.y;
                Jloc += wPe * rPf * rPf + wQe * rQf * rQf;
                const double Vi = bV[qi], Vj = bV[qj];
                const double g_ = T.end_g[ee], b_ = T.end_b[ee], bh_ = T.end_bh[ee];
                const double2 tr = end_trig(bC[qi], bS[qi], bC[qj], bS[qj], g_, b_);
                const double gc_bs = tr.x, gs_bc = tr.y;
                const double ViVj = Vi * Vj;
                // partials w.r.t. (Vi, thi, Vj, thj)
                double dP[4], dQ[4];
                dP[0] = 2.0 * Vi * g_ - Vj * gc_bs;
                dP[1] = ViVj * gs_bc;
                dP[2] = -Vi * gc_bs;
                dP[3] = -dP[1];
                dQ[0] = -2.0 * Vi * (b_ + bh_) - Vj * gs_bc;
                dQ[1] = -ViVj * gc_bs;
                dQ[2] = -Vi * gs_bc;
                dQ[3] = -dQ[1];
                o = T.end_own[ee];
                const double2 ij = inj[o];
                const double aP = wPe * rPf + ij.x, aQ = wQe * rQf + ij.y;
                const int *vv = T.end_var + 4 * (long long)ee;
                gv0 = vv[0];
                gv1 = vv[1];
                own_g[0] = aP * dP[0] + aQ * dQ[0];
                own_g[1] = aP * dP[1] + aQ * dQ[1];
#pragma unroll
                for (int a = 2; a < 4; ++a) {
                    const int v = vv[a];
                    if (v >= 0) atomicAdd(g + v, aP * dP[a] + aQ * dQ[a]);
                }
                RG hP[4], hQ[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    hP[a] = RG(dP[a]);
                    hQ[a] = RG(dQ[a]);
                }
                const RG wp = RG(wPe), wq = RG(wQe);
                const int *gp = T.end_gpos + 10 * (long long)ee;
                int idx = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = a; c < 4; ++c, ++idx) {
                        const RG v = wp * hP[a] * hP[c] + wq * hQ[a] * hQ[c];
                        if (idx == 0) { own_s[0] = v; gp0 = gp[0]; }
                        else if (idx == 1) { own_s[1] = v; gp1 = gp[1]; }
                        else if (idx == 4) { own_s[2] = v; gp4 = gp[4]; }
                        else {
                            const int p = gp[idx];
                            if (p >= 0) atomicAdd(st + p, v);
                        }
                    }
                // injection partials: own-bus part summed per bus, neighbour part kept per end
                own_s[3] = hP[0];
                own_s[4] = hP[1];
                own_s[5] = hQ[0];
                own_s[6] = hQ[1];
                RG *nb = (RG *)(endbuf + (size_t)e * endstride);
                nb[0] = hP[2];
                nb[1] = hP[3];
                nb[2] = hQ[2];
                nb[3] = hQ[3];
            }
            // runs of one owning bus: heads and each lane's run end
            const int kprev = __shfl_up_sync(FULL, o, 1);
            const bool head = lane == 0 || kprev != o;
            const unsigned heads = __ballot_sync(FULL, head);
            const unsigned later = lane == 31 ? 0u : (heads & (0xFFFFFFFEu << lane));
            const int run_end = later ? __ffs(later) - 2 : 31;
            const int longest = (int)__reduce_max_sync(FULL, (unsigned)(run_end - lane + 1));
            for (int d = 1; d < longest; d <<= 1) {
                const bool take = lane + d <= run_end;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const double t = __shfl_down_sync(FULL, own_g[q], d);
                    if (take) own_g[q] += t;
                }
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const RG t = __shfl_down_sync(FULL, own_s[q], d);
                    if (take) own_s[q] += t;
                }
            }
            if (valid && head) {
                if (gv0 >= 0) atomicAdd(g + gv0, own_g[0]);
                if (gv1 >= 0) atomicAdd(g + gv1, own_g[1]);
                if (gp0 >= 0) atomicAdd(st + gp0, own_s[0]);
                if (gp1 >= 0) atomicAdd(st + gp1, own_s[1]);
                if (gp4 >= 0) atomicAdd(st + gp4, own_s[2]);
#pragma unroll
                for (int q = 0; q < 4; ++q) atomicAdd(self + 4 * o + q, own_s[3 + q]);
            }
        }
    }
    __syncthreads();
    // ---- E4: injection-row gain terms, one item per pair of buses in the row
    for (int it = tid; it < A.n_items; it += nt) {
        const int ii = A.item_base + it;
        const int4 rec = T.item_rec[ii];
        const int4 pos = reinterpret_cast<const int4 *>(T.item_pos)[ii];
        const int o = rec.x, eu = rec.y, ev = rec.z;
        const int cu = rec.w & 0xffff, cv = rec.w >> 16;
        RG pu[4], pv[4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int eb = t == 0 ? eu : ev, ec = t == 0 ? cu : cv;
            RG *dst = t == 0 ? pu : pv;
            if (eb < 0) {
#pragma unroll
                for (int a = 0; a < 4; ++a) dst[a] = self[4 * o + a];
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) dst[a] = RG(0);
                for (int e = eb; e < eb + ec; ++e) {
                    const RG *nb = (const RG *)(endbuf + (size_t)e * endstride);
#pragma unroll
                    for (int a = 0; a < 4; ++a) dst[a] += nb[a];
                }
            }
        }
        // pu = (dP/dV_u, dP/dth_u, dQ/dV_u, dQ/dth_u)
        const RG wp = RG(wt(rP + o)), wq = RG(wt(rQ + o));
        const int p4[4] = {pos.x, pos.y, pos.z, pos.w};
        const bool u_eq_v = eu == ev;
        if (u_eq_v) {
            atomicAdd(st + p4[0], wp * pu[0] * pu[0] + wq * pu[2] * pu[2]);
            if (p4[1] >= 0) atomicAdd(st + p4[1], wp * pu[1] * pu[0] + wq * pu[3] * pu[2]);
            if (p4[2] >= 0) atomicAdd(st + p4[2], wp * pu[1] * pu[1] + wq * pu[3] * pu[3]);
        } else {
            atomicAdd(st + p4[0], wp * pu[0] * pv[0] + wq * pu[2] * pv[2]);
            if (p4[1] >= 0) atomicAdd(st + p4[1], wp * pu[0] * pv[1] + wq * pu[2] * pv[3]);
            if (p4[2] >= 0) atomicAdd(st + p4[2], wp * pu[1] * pv[0] + wq * pu[3] * pv[2]);
            if (p4[3] >= 0) atomicAdd(st + p4[3], wp * pu[1] * pv[1] + wq * pu[3] * pv[3]);
        }
    }
    __syncthreads();
    // ---- rhs in solve precision
    for (int i = tid; i < nv; i += nt) y[i] = RS(g[i]);
    __syncthreads();
    // ---- Schur-mode factorisation (Sec. 4.3): leaves S_b and b_hat in the trailing block
    factor_tasks<RG, RS>(A.F, T, FlatStore<RG>{st}, y, ctr, &s_err);
    // ---- outputs
    if (A.in_smem) {
        RG *dst = fac + A.fac_base + (long long)s * A.fac_stride;
        for (int i = tid; i < A.F.store_total; i += nt) dst[i] = st[i];
    }
    RS *cdst = cvec + A.c_base + (long long)s * A.F.n_int;
    for (int i = tid; i < A.F.n_int; i += nt) cdst[i] = y[i];
    double *bdst = bh + A.bh_base + (long long)s * A.F.n_bnd;
    for (int i = tid; i < A.F.n_bnd; i += nt) bdst[i] = double(y[A.F.n_int + i]);
    const double Js = block_sum(Jloc, red);
    if (tid == 0) {
        atomicAdd(X.J + s, Js);
        if (s_err) atomicOr(X.err + s, s_err);
    }
    clk_end(X.clk);
}

// ---------------------------------------------------------------------------
// coordinator: assembly (Eq. global_assembly), sparse Cholesky, FP64 refinement
// ---------------------------------------------------------------------------
struct BndDev {
    FacDev F;
    int n_gamma;
    const int *asm_beg, *asm_area, *asm_off;
    const int *rhs_beg, *rhs_area, *rhs_lv;
    const int *bvar_ibus, *bvar_isT;
    const long long *asm_abs, *rhs_abs;   // absolute gather sources for snapshot 0
    const int *asm_str, *rhs_str;         // their per-snapshot strides
    long long stride;     // storage elements per snapshot
    int split;            // storage entries from here on live in shared memory
    int smem_off_ctr;     // byte offset of the task counters (2 nsn + 1 ints)
    int split_cl;         // 2-block cluster: entries [split_cl, ...) in block 0, the rest in block 1
    int smem_off_st;      // byte offset of the shared part of the storage
};

// Gathers S_Gamma = sum_k E_k^T S_b^k E_k (Eq. global_assembly) into the
// boundary factor storage (and the refinement's copy Am when given): entry P
// sums the stored S_b entries listed in asm_beg[P] .. asm_beg[P+1].  Four
// entries per thread at a time, so that their first source loads overlap.
template <class RG, class ST>
__device__ __forceinline__ void assemble_boundary(const BndDev &B, const RG *__restrict__ fac, int s,
                                                  const ST &st, RG *Am, int t0, int nt) {
    const long long so = (long long)s;
    for (int P0 = t0; P0 < B.F.store_total; P0 += 4 * nt) {
        int i0[4], i1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int P = P0 + u * nt;
            const bool ok = P < B.F.store_total;
            i0[u] = ok ? B.asm_beg[P] : 0;
            i1[u] = ok ? B.asm_beg[P + 1] : 0;
        }
        RG v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = i0[u] < i1[u] ? fac[B.asm_abs[i0[u]] + so * B.asm_str[i0[u]]] : RG(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            for (int i = i0[u] + 1; i < i1[u]; ++i) v[u] += fac[B.asm_abs[i] + so * B.asm_str[i]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int P = P0 + u * nt;
            if (P < B.F.store_total) {
                *st.at(P) = v[u];
                if (Am) Am[P] = v[u];
            }
        }
    }
}

// r -= S x for the boundary system S (symmetric, lower part stored in
// supernode layout, FP32 or FP64 values, FP64 accumulation): one task per
// diagonal block and per 32-row chunk below it, spread over the team's warps.
// A chunk (lane = row) adds its rows' products in registers and the column
// sums by a transpose-reduction of the 32 per-lane columns (31 exchanges).
template <class RG>
__device__ __noinline__ void residual_chunk(const RG *P, int w, int ld, int row0, int c0,
                                            const int *rws, const double *x, double *r) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, row = row0 + lane;
    const bool ok = row < ld;
    const int grow = ok ? rws[row - w] : 0;
    const double xr = ok ? x[grow] : 0.0;
    double v[32];
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const double a = (ok && c < w) ? double(P[(size_t)c * ld + row]) : 0.0;
        acc += a * (c < w ? x[c0 + c] : 0.0);
        v[c] = a * xr;
    }
    if (ok) atomicAdd(r + grow, -acc);
    // after the exchange at distance d a lane keeps the half of its columns
    // whose bit d matches its own; in the end lane c holds column c's sum
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const bool up = (lane & d) != 0;
#pragma unroll
        for (int k = 0; k < d; ++k) {
            const double send = up ? v[k] : v[k + d];
            const double keep = up ? v[k + d] : v[k];
            v[k] = keep + __shfl_xor_sync(FULL, send, d);
        }
    }
    if (lane < w) atomicAdd(r + c0 + lane, -v[0]);
}

template <class RG, class TM>
__device__ void boundary_residual(const FacDev &F, const Tables &T, const RG *Am, const double *x,
                                  double *r, const TM &tm) {
    const int lane = threadIdx.x & 31;
    const int4 *crec = T.chunk_rec + 2 * (long long)F.chunk_base;
    const int nch = T.lev_chunks[F.levchunk_base + F.nlev];
    const int *rows = T.rows + F.rows_base;
    for (int k = tm.warp(); k < F.nsn + nch; k += tm.nwarps()) {
        if (k < F.nsn) {
            const int sg = F.sn_base + k;
            const int w = T.sn_w[sg], ld = w + T.sn_nr[sg], c0 = T.sn_c0[sg];
            const RG *P = Am + T.sn_off[sg];
            if (lane < w) {
                double acc = 0.0;
                for (int c = 0; c < w; ++c) {
                    const RG a = c <= lane ? P[(size_t)c * ld + lane] : P[(size_t)lane * ld + c];
                    acc += double(a) * x[c0 + c];
                }
                atomicAdd(r + c0 + lane, -acc);
            }
        } else {
            const int4 q = crec[2 * (k - F.nsn)], q2 = crec[2 * (k - F.nsn) + 1];
            residual_chunk<RG>(Am + q.x, q.y, q.z, q.w, q2.x, rows + q2.y, x, r);
        }
    }
}

template <class RG, class RS>
__global__ void __launch_bounds__(512) k_boundary(const AreaDev *__restrict__ areas, Tables T,
                                                  State X, BndDev B, const RG *__restrict__ fac,
                                                  const double *__restrict__ bh, RG *bst, RG *bA,
                                                  double *dxG, int refine) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_err;
    const int s = blockIdx.x;
    if (!X.active[s]) return;
    clk_begin(X.clk);
    const int tid = threadIdx.x, nt = blockDim.x, nG = B.n_gamma;
    double *bhat = (double *)smem;
    double *x = bhat + nG;
    double *r = x + nG;
    RS *y = (RS *)(r + nG);
    // the top of the elimination tree (most updates) in shared memory, the rest in global
    const SplitStore<RG> st{bst + (long long)s * B.stride, (RG *)(smem + B.smem_off_st), B.split};
    RG *Am = bA + (long long)s * B.stride;
    if (tid == 0) s_err = 0;
    assemble_boundary<RG>(B, fac, s, st, refine ? Am : nullptr, tid, nt);
    for (int gi = tid; gi < nG; gi += nt) {
        double v = 0.0;
        for (int i = B.rhs_beg[gi]; i < B.rhs_beg[gi + 1]; ++i)
            v += bh[B.rhs_abs[i] + (long long)s * B.rhs_str[i]];
        bhat[gi] = v;
        y[gi] = RS(v);
    }
    __syncthreads();
    factor_numeric<RG, RS>(B.F, T, st, y, (int *)(smem + B.smem_off_ctr), &s_err);
    back_solve<RG, RS>(B.F, T, st, y);
    for (int gi = tid; gi < nG; gi += nt) x[gi] = double(y[gi]);
    __syncthreads();
    for (int it = 0; it < refine; ++it) {
        // r = b_hat - S_Gamma x, FP64 accumulation over the stored lower triangle
        for (int gi = tid; gi < nG; gi += nt) r[gi] = bhat[gi];
        __syncthreads();
        boundary_residual<RG>(B.F, T, Am, x, r, BlockTeam());
        __syncthreads();
        for (int gi = tid; gi < nG; gi += nt) y[gi] = RS(r[gi]);
        __syncthreads();
        solve_forward<RG, RS>(B.F, T, st, y);
        back_solve<RG, RS>(B.F, T, st, y);
        for (int gi = tid; gi < nG; gi += nt) x[gi] += double(y[gi]);
        __syncthreads();
    }
    double mx = 0.0;
    bool bad = false;
    for (int gi = tid; gi < nG; gi += nt) {
        const double d = x[gi];
        dxG[(long long)s * nG + gi] = d;
        const long long at = (long long)s * X.N + B.bvar_ibus[gi];
        if (B.bvar_isT[gi]) X.xT[at] += d;
        else X.xV[at] += d;
        if (!isfinite(d)) bad = true;
        mx = fmax(mx, fabs(d));
    }
    if (bad) atomicOr(X.err + s, 2);
    mx = block_max(mx, red);
    if (tid == 0) {
        atomicMax(X.maxstep + s, (unsigned long long)__double_as_longlong(mx));
        if (s_err) atomicOr(X.err + s, s_err);
    }
    clk_end(X.clk);
}

// The coordinator for one snapshot on a 2-block cluster: the boundary
// factor lives in the shared memory of both blocks (distributed shared
// memory), the vectors in block 0's; both blocks' warps share the level
// schedule, with cluster barriers between task groups.
template <class RG, class RS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512)
    k_boundary_cl(Tables T, State X, BndDev B, const RG *__restrict__ fac,
                  const double *__restrict__ bh, RG *bA, double *dxG, int refine) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_err;
    const int rank = (int)__clusterRelativeBlockRank();
    const int s = blockIdx.x >> 1;
    if (!X.active[s]) return;   // both blocks of the cluster leave together
    clk_begin(X.clk);
    const ClusterTeam tm{rank};
    const int tid = threadIdx.x, nt = blockDim.x, nG = B.n_gamma;
    const int ct = rank * nt + tid, cn = 2 * nt;
    if (tid == 0) s_err = 0;
    tm.sync();   // both blocks are running before either touches the other's memory
    unsigned char *sm0 = (unsigned char *)__cluster_map_shared_rank(smem, 0);
    unsigned char *sm1 = (unsigned char *)__cluster_map_shared_rank(smem, 1);
    double *bhat = (double *)sm0;
    double *x = bhat + nG;
    double *r = x + nG;
    RS *y = (RS *)(r + nG);
    const ClusterStore<RG> st{(RG *)(sm0 + B.smem_off_st), (RG *)sm1, B.split_cl};
    RG *Am = bA + (long long)s * B.stride;
    assemble_boundary<RG>(B, fac, s, st, refine ? Am : nullptr, ct, cn);
    for (int gi = ct; gi < nG; gi += cn) {
        double v = 0.0;
        for (int i = B.rhs_beg[gi]; i < B.rhs_beg[gi + 1]; ++i)
            v += bh[B.rhs_abs[i] + (long long)s * B.rhs_str[i]];
        bhat[gi] = v;
        y[gi] = RS(v);
    }
    tm.sync();
    factor_levels<RG, RS>(B.F, T, st, y, &s_err, tm);
    back_solve<RG, RS>(B.F, T, st, y, tm);
    for (int gi = ct; gi < nG; gi += cn) x[gi] = double(y[gi]);
    tm.sync();
    for (int it = 0; it < refine; ++it) {
        // r = b_hat - S_Gamma x, FP64 accumulation over the stored lower triangle
        for (int gi = ct; gi < nG; gi += cn) r[gi] = bhat[gi];
        tm.sync();
        boundary_residual<RG>(B.F, T, Am, x, r, tm);
        tm.sync();
        for (int gi = ct; gi < nG; gi += cn) y[gi] = RS(r[gi]);
        tm.sync();
        solve_forward<RG, RS>(B.F, T, st, y, tm);
        back_solve<RG, RS>(B.F, T, st, y, tm);
        for (int gi = ct; gi < nG; gi += cn) x[gi] += double(y[gi]);
        tm.sync();
    }
    double mx = 0.0;
    bool bad = false;
    for (int gi = ct; gi < nG; gi += cn) {
        const double d = x[gi];
        dxG[(long long)s * nG + gi] = d;
        const long long at = (long long)s * X.N + B.bvar_ibus[gi];
        if (B.bvar_isT[gi]) X.xT[at] += d;
        else X.xV[at] += d;
        if (!isfinite(d)) bad = true;
        mx = fmax(mx, fabs(d));
    }
    if (bad) atomicOr(X.err + s, 2);
    mx = block_max(mx, red);
    if (tid == 0) {
        atomicMax(X.maxstep + s, (unsigned long long)__double_as_longlong(mx));
        if (s_err) atomicOr(X.err + s, s_err);
    }
    tm.sync();   // neither block leaves while the other may still use its shared memory
    clk_end(X.clk);
}

// ---------------------------------------------------------------------------
// back-substitution (Eq. backsub) + state update (FP64)
// ---------------------------------------------------------------------------
template <class RG, class RS>
__global__ void __launch_bounds__(512) k_back(const AreaDev *__restrict__ areas, Tables T, State X,
                                              const int2 *__restrict__ inst, int area_only,
                                              const RG *__restrict__ fac, const RS *__restrict__ cvec,
                                              const double *__restrict__ dxG, int n_gamma) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    int k, s;
    if (area_only >= 0) {
        k = area_only;
        s = blockIdx.x;
    } else {
        const int2 ks = inst[blockIdx.x];
        k = ks.x;
        s = ks.y;
    }
    if (!X.active[s]) return;
    clk_begin(X.clk);
    const AreaDev A = areas[k];
    const int tid = threadIdx.x, nt = blockDim.x;
    RS *y = (RS *)smem;
    // each factor entry is read once, straight from global memory: many small
    // blocks per SM hide the latency better than staging the factor on chip
    const RG *fst = fac + A.fac_base + (long long)s * A.fac_stride;
    const RS *c = cvec + A.c_base + (long long)s * A.F.n_int;
    for (int i = tid; i < A.F.n_int; i += nt) y[i] = c[i];
    for (int lv = tid; lv < A.F.n_bnd; lv += nt)
        y[A.F.n_int + lv] = RS(dxG[(long long)s * n_gamma + T.ebnd[A.ebnd_base + lv]]);
    __syncthreads();
    back_solve<RG, RS>(A.F, T, FlatStore<const RG>{fst}, y);
    double mx = 0.0;
    bool bad = false;
    for (int q = tid; q < A.nb_int; q += nt) {
        const long long at = (long long)s * X.N + T.locbus[A.bus_base + q];
        const double dV = double(y[T.qvarV[A.bus_base + q]]);
        X.xV[at] += dV;
        mx = fmax(mx, fabs(dV));
        bad |= !isfinite(dV);
        const int vt = T.qvarT[A.bus_base + q];
        if (vt >= 0) {
            const double dT = double(y[vt]);
            X.xT[at] += dT;
            mx = fmax(mx, fabs(dT));
            bad |= !isfinite(dT);
        }
    }
    if (bad) atomicOr(X.err + s, 2);
    mx = block_max(mx, red);
    if (tid == 0) atomicMax(X.maxstep + s, (unsigned long long)__double_as_longlong(mx));
    clk_end(X.clk);
}

// layout conversions (defined below, in the translation unit that includes
// this header without MASE_SHARED_TEMPLATES_ONLY)
__global__ void k_gather_rows(const double *__restrict__ src, double *__restrict__ dst,
                              const int *__restrict__ perm, int M, int S);
__global__ void k_gather_mask(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                              const int *__restrict__ perm, int M, int S);
__global__ void k_state_in(const double *__restrict__ x, double *xV, double *xT,
                           const int *__restrict__ bus_of_ibus, int N, int S, int flat);
__global__ void k_state_out(double *__restrict__ x, const double *xV, const double *xT,
                            const int *__restrict__ bus_of_ibus, int N, int S);

#ifndef MASE_SHARED_TEMPLATES_ONLY
// ---------------------------------------------------------------------------
// objective J = r^T W r at the current states (Eq. wls), per snapshot
// ---------------------------------------------------------------------------
// One block per (area, snapshot) evaluates the area's rows: voltage rows,
// flow rows at every owned branch end and injection rows as sums of those
// flows.  Shared memory holds only the bus values and the end flows
// (AreaDev::obj_smem_bytes), so several blocks share an SM.
template <bool VG>
__global__ void __launch_bounds__(256) k_objective(const AreaDev *__restrict__ areas, Tables T, State X,
                                                   const int2 *__restrict__ inst, unsigned char *vscratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    const int2 ks = inst[blockIdx.x];
    const int k = ks.x, s = ks.y;
    const AreaDev A = areas[k];
    const int tid = threadIdx.x, nt = blockDim.x;
    unsigned char *vb = (VG && A.vec_global) ? vscratch + A.vec_base + (long long)s * A.vec_stride : smem;
    double *bV = (double *)vb;
    double *bC = bV + A.nb_loc;
    double *bS = bC + A.nb_loc;
    double2 *pq = (double2 *)(vb + A.obj_off_end);
    const long long zb = (long long)s * X.M + A.zrow_base;
    const double *z = X.z + zb;
    const double *Wr = X.W + A.zrow_base;
    const uint8_t *mk = X.mask ? X.mask + zb : nullptr;
    auto wt = [&](int r) { return mk ? (mk[r] ? Wr[r] : 0.0) : Wr[r]; };
    const int n_own = A.n_own, n_ends = A.n_ends;
    const int rP = n_own, rQ = 2 * n_own, rPe = 3 * n_own, rQe = 3 * n_own + n_ends;
    for (int q = tid; q < A.nb_loc; q += nt) {
        const int ib = T.locbus[A.bus_base + q];
        double sn, cs;
        sincos(X.xT[(long long)s * X.N + ib], &sn, &cs);
        bV[q] = X.xV[(long long)s * X.N + ib];
        bC[q] = cs;
        bS[q] = sn;
    }
    __syncthreads();
    double Jloc = 0.0;
    for (int e = tid; e < n_ends; e += nt) {
        const int ee = A.end_base + e;
        const int qi = T.end_qi[ee], qj = T.end_qj[ee];
        const EndFlow f = end_flow(bV[qi], bV[qj], bC[qi], bS[qi], bC[qj], bS[qj], T.end_g[ee],
                                   T.end_b[ee], T.end_bh[ee]);
        pq[e] = make_double2(f.P, f.Q);
        const double rPf = z[rPe + e] - f.P, rQf = z[rQe + e] - f.Q;
        Jloc += wt(rPe + e) * rPf * rPf + wt(rQe + e) * rQf * rQf;
    }
    __syncthreads();
    for (int o = tid; o < n_own; o += nt) {
        const int q = T.own_q[A.own_base + o];
        const double rv = z[o] - bV[q];
        double Pi = 0.0, Qi = 0.0;
        for (int e = T.own_ebeg[A.own1_base + o]; e < T.own_ebeg[A.own1_base + o + 1]; ++e) {
            Pi += pq[e].x;
            Qi += pq[e].y;
        }
        const double rp = z[rP + o] - Pi, rq = z[rQ + o] - Qi;
        Jloc += wt(o) * rv * rv + wt(rP + o) * rp * rp + wt(rQ + o) * rq * rq;
    }
    const double Js = block_sum(Jloc, red);
    if (tid == 0) atomicAdd(X.J + s, Js);
}

// ---------------------------------------------------------------------------
// per-snapshot bookkeeping after a step
// ---------------------------------------------------------------------------
// Per-step clocks and loop control, kept on the device so that a solve can
// run as one graph with a device-side loop.
struct StepCtl {
    unsigned long long *clk;   // [3][2] stage clocks of the area, coordinator and back kernels
    double *acc;               // [4] ms summed over the solve: area, coordinator, back, bookkeeping
    int *steps;                // Gauss-Newton steps run in this solve
    int *n_active;             // snapshots still iterating after the last step
};

__global__ void k_finalize(State X, int *iters, int *status, double *laststep,
                           const StopRule *__restrict__ rule, StepCtl ctl,
                           cudaGraphConditionalHandle cond, int use_cond) {
    const unsigned long long t0 = gtimer();
    const double tol = rule->tol;
    const int max_iter = rule->max_iter;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int s = threadIdx.x; s < X.S; s += blockDim.x) {
        if (X.active[s]) {
            const int it = ++iters[s];
            const double m = __longlong_as_double((long long)X.maxstep[s]);
            laststep[s] = m;
            const int e = X.err[s];
            int st = -1;
            if (e & 4) st = 4;                       // MASE_SNAP_DEVICE (bounded wait gave up)
            else if (e & 1) st = 2;                  // MASE_SNAP_NOT_SPD
            else if ((e & 2) || !isfinite(m)) st = 3; // MASE_SNAP_NONFINITE
            else if (m < tol) st = 0;                 // MASE_SNAP_CONVERGED
            else if (it >= max_iter) st = 1;          // MASE_SNAP_MAX_ITER
            if (st >= 0) {
                status[s] = st;
                X.active[s] = 0;
            } else {
                ++c;
            }
        }
        X.maxstep[s] = 0ull;
        X.J[s] = 0.0;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        *ctl.n_active = cnt;
        const int steps = ++*ctl.steps;
        for (int i = 0; i < 3; ++i) {
            const unsigned long long a = ctl.clk[2 * i], b = ctl.clk[2 * i + 1];
            if (b > a) ctl.acc[i] += 1e-6 * double(b - a);
            ctl.clk[2 * i] = ~0ull;
            ctl.clk[2 * i + 1] = 0ull;
        }
        if (use_cond) cudaGraphSetConditional(cond, (cnt > 0 && steps < max_iter) ? 1u : 0u);
        ctl.acc[3] += 1e-6 * double(gtimer() - t0);
    }
}

// clears the step norm and the objective left by inner local iterations
__global__ void k_clear_step(State X) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < X.S; s += gridDim.x * blockDim.x) {
        X.maxstep[s] = 0ull;
        X.J[s] = 0.0;
    }
}

__global__ void k_reset(State X, int *iters, int *status, double *laststep, StepCtl ctl) {
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        if (threadIdx.x < 6) ctl.clk[threadIdx.x] = (threadIdx.x & 1) ? 0ull : ~0ull;
        if (threadIdx.x < 4) ctl.acc[threadIdx.x] = 0.0;
        if (threadIdx.x == 0) *ctl.steps = 0;
    }
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < X.S; s += gridDim.x * blockDim.x) {
        X.active[s] = 1;
        X.err[s] = 0;
        X.J[s] = 0.0;
        X.maxstep[s] = 0ull;
        iters[s] = 0;
        status[s] = 1;
        laststep[s] = 0.0;
    }
}

// Flat-start fallback of the learned start: every snapshot flagged in
// `restart` goes back to Vm = 1, Va = 0 with a fresh iteration count and is
// the only kind left active; the step counter of the loop starts again.
__global__ void k_restart(State X, int *iters, int *status, double *laststep, const int *restart,
                          StepCtl ctl) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctl.steps = 0;
    const long long n = (long long)X.N * X.S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / X.N;
        if (!restart[s]) continue;
        X.xV[i] = 1.0;
        X.xT[i] = 0.0;
        if (i - s * X.N == 0) {
            X.active[s] = 1;
            X.err[s] = 0;
            X.J[s] = 0.0;
            X.maxstep[s] = 0ull;
            iters[s] = 0;
            status[s] = 1;
            laststep[s] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// layout conversions
// ---------------------------------------------------------------------------
__global__ void k_gather_rows(const double *__restrict__ src, double *__restrict__ dst,
                              const int *__restrict__ perm, int M, int S) {
    const long long n = (long long)M * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / M;
        const int r = (int)(i - s * M);
        dst[i] = src[s * M + perm[r]];
    }
}
__global__ void k_gather_mask(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                              const int *__restrict__ perm, int M, int S) {
    const long long n = (long long)M * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / M;
        const int r = (int)(i - s * M);
        dst[i] = src[s * M + perm[r]];
    }
}
// canonical x[s][2N] <-> internal (xV, xT)[s][N]
__global__ void k_state_in(const double *__restrict__ x, double *xV, double *xT,
                           const int *__restrict__ bus_of_ibus, int N, int S, int flat) {
    const long long n = (long long)N * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / N;
        const int ib = (int)(i - s * N);
        if (flat) {
            xV[i] = 1.0;
            xT[i] = 0.0;
        } else {
            const int b = bus_of_ibus[ib];
            xV[i] = x[s * 2 * N + b];
            xT[i] = x[s * 2 * N + N + b];
        }
    }
}
__global__ void k_state_out(double *__restrict__ x, const double *xV, const double *xT,
                            const int *__restrict__ bus_of_ibus, int N, int S) {
    const long long n = (long long)N * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / N;
        const int ib = (int)(i - s * N);
        const int b = bus_of_ibus[ib];
        x[s * 2 * N + b] = xV[i];
        x[s * 2 * N + N + b] = xT[i];
    }
}

// h(x) in canonical order (Eq. typed_meas), one thread per bus or branch.
__global__ void k_measure(const double *__restrict__ x, double *__restrict__ z, int N, int L, int S,
                          const int *__restrict__ from, const int *__restrict__ to,
                          const double *__restrict__ g, const double *__restrict__ b,
                          const double *__restrict__ bh, const int *__restrict__ inc_beg,
                          const int *__restrict__ inc_br) {
    const int M = 3 * N + 4 * L;
    const long long n = (long long)(N + L) * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / (N + L);
        const int u = (int)(i - s * (N + L));
        const double *Vm = x + s * 2 * N;
        const double *Va = Vm + N;
        double *zs = z + s * M;
        if (u < N) {
            double P = 0.0, Q = 0.0, si, ci;
            sincos(Va[u], &si, &ci);
            for (int t = inc_beg[u]; t < inc_beg[u + 1]; ++t) {
                const int l = inc_br[t];
                const int j = from[l] == u ? to[l] : from[l];
                double sj, cj;
                sincos(Va[j], &sj, &cj);
                const EndFlow f = end_flow(Vm[u], Vm[j], ci, si, cj, sj, g[l], b[l], bh[l]);
                P += f.P;
                Q += f.Q;
            }
            zs[u] = Vm[u];
            zs[N + u] = P;
            zs[2 * N + u] = Q;
        } else {
            const int l = u - N;
            const int f_ = from[l], t_ = to[l];
            double sf, cf, stt, ct;
            sincos(Va[f_], &sf, &cf);
            sincos(Va[t_], &stt, &ct);
            const EndFlow a = end_flow(Vm[f_], Vm[t_], cf, sf, ct, stt, g[l], b[l], bh[l]);
            const EndFlow c = end_flow(Vm[t_], Vm[f_], ct, stt, cf, sf, g[l], b[l], bh[l]);
            zs[3 * N + l] = a.P;
            zs[3 * N + L + l] = a.Q;
            zs[3 * N + 2 * L + l] = c.P;
            zs[3 * N + 3 * L + l] = c.Q;
        }
    }
}

#endif  // MASE_SHARED_TEMPLATES_ONLY

}  // namespace mase_dev
