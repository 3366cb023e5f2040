// C-ABI implementation of libmase (see include/mase.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mase.h"
#include "internal.h"
#include "kernels.cuh"
#include "setup.h"

using namespace mase_dev;

namespace {

// the back-substitution is a gather over a few warps' worth of rows per
// level; 256 threads measured faster than 512 on the 9241-bus workload
constexpr int kBackThreads = 256;
// shared memory of one SM that blocks can use (228 KB, less 1 KB each)
constexpr size_t kSmemPerSM = 228 * 1024;
// narrowest source panel whose update units run on the tensor cores (MIXED)
constexpr int kDefaultTensorUnits = 0;

thread_local std::string g_last_error;

int set_err(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(MASE_EDEVICE, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)


template <class V>
void app(V &dst, const V &src) {
    dst.insert(dst.end(), src.begin(), src.end());
}

FacDev append_fac(HostTables &H, const mase::SymFactor &F) {
    FacDev d{};
    d.n_int = F.n_int;
    d.n_bnd = F.n_bnd;
    d.nsn = F.nsn();
    d.nlev = F.nlev();
    d.store_int = F.store_int;
    d.store_total = F.store_total;
    d.off_B = F.off_B;
    d.max_w = F.max_w;
    d.sn_base = (int)H.sn_c0.size();
    app(H.sn_c0, F.sn_c0);
    app(H.sn_w, F.sn_w);
    app(H.sn_nr, F.sn_nr);
    app(H.sn_off, F.sn_off);
    app(H.sn_order, F.sn_order);
    d.levoff_base = (int)H.lev_off.size();
    if (F.lev_off.empty()) H.lev_off.push_back(0);
    else app(H.lev_off, F.lev_off);
    d.rows_base = (int)H.rows.size();
    app(H.rows, F.rows);
    d.rel_base = (int)H.rel.size();
    app(H.rel, F.rel);
    d.task_base = (int)(H.tasks.size() / 16);
    d.n_tasks = F.n_tasks;
    app(H.tasks, F.tasks);
    d.level_sched = F.level_sched;
    d.levtask_base = (int)H.lev_tasks.size();
    app(H.lev_tasks, F.lev_tasks);
    d.chunk_base = (int)H.chunk_rec.size() / 8;
    app(H.chunk_rec, F.chunk_rec);
    d.levchunk_base = (int)H.lev_chunks.size();
    if (F.lev_chunks.empty()) H.lev_chunks.push_back(0);
    else app(H.lev_chunks, F.lev_chunks);
    return d;
}



bool is_device_ptr(const void *p) { return mase_internal::is_device_pointer(p); }

}  // namespace

bool mase_internal::is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {

}  // namespace


namespace {

// The library works on its own non-blocking stream; every call first waits
// for work already queued on the caller's stream and, before returning,
// makes the caller's stream wait for the library's work.
int join_in(mase_handle *h) {
    CK(cudaEventRecord(h->ev_in, h->user_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
    return MASE_OK;
}
int join_out(mase_handle *h) {
    CK(cudaEventRecord(h->ev_out, h->stream));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
    return MASE_OK;
}

template <class RG, class RS>
void setup_attrs(mase_handle *h) {
    cudaFuncSetAttribute(k_local<RG, RS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_limit);
    cudaFuncSetAttribute(k_local<RG, RS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_limit);
    cudaFuncSetAttribute(k_back<RG, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_limit);
    cudaFuncSetAttribute(k_boundary<RG, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         h->smem_limit);
    cudaFuncSetAttribute(k_boundary_cl<RG, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         h->smem_limit);
    cudaFuncSetAttribute(k_objective<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_limit);
    cudaFuncSetAttribute(k_objective<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_limit);
}

State make_state(mase_handle *h) {
    State X;
    X.N = h->S.N;
    X.M = h->S.m;
    X.S = h->n_snap;
    X.xV = h->xV.p;
    X.xT = h->xT.p;
    X.z = h->z_int.p;
    X.W = h->W.p;
    X.mask = h->has_mask ? h->mask_int.p : nullptr;
    X.active = h->active.p;
    X.err = h->err.p;
    X.J = h->J.p;
    X.maxstep = h->maxstep.p;
    X.clk = nullptr;
    return X;
}

StepCtl make_ctl(mase_handle *h) {
    StepCtl c;
    c.clk = h->clk.p;
    c.acc = h->clk_acc.p;
    c.steps = h->steps_dev.p;
    c.n_active = h->n_active.p;
    return c;
}

// One Gauss-Newton step for every active snapshot: local condensation,
// coordinator, back-substitution, bookkeeping.  Each stage's kernels carry a
// device clock (first block start, last block end), which the bookkeeping
// kernel sums per step, so stage times need no host events and also hold
// inside a graph with a device-side loop.  With options.profile the host
// steps the loop and CUDA events bracket the stages as well.
inline void mark(mase_handle *h, int i) {
    if (h->opt.profile) cudaEventRecord(h->ev_stage[i], h->stream);
}

template <class RG, class RS>
void launch_class(mase_handle *h, const State &X, RG *fac, RS *cv, const LocalClass &c, cudaStream_t st) {
    auto kern = h->vec_global ? k_local<RG, RS, true> : k_local<RG, RS, false>;
    kern<<<(int)c.inst_h.size(), c.threads, c.smem, st>>>(h->d_areas.p, h->T, X, c.inst.p, -1, fac, cv,
                                                         h->bh.p, h->vscratch.p);
}

// The area kernel over every (area, snapshot): one launch per class, the
// classes on forked streams so that they share the GPU.
template <class RG, class RS>
void launch_local(mase_handle *h, const State &X, RG *fac, RS *cv, int *launches) {
    const int S = h->n_snap, K = h->S.K, nt = h->threads;
    auto kern = h->vec_global ? k_local<RG, RS, true> : k_local<RG, RS, false>;
    unsigned char *vs = h->vscratch.p;
    if (h->opt.schedule == MASE_BATCHED) {
        const int nc = (int)h->lcls.size();
        if (nc > 1) {
            cudaEventRecord(h->ev_fork, h->stream);
            for (int c = 1; c < nc; ++c) {
                cudaStreamWaitEvent(h->side[c - 1], h->ev_fork, 0);
                launch_class<RG, RS>(h, X, fac, cv, *h->lcls[c], h->side[c - 1]);
                cudaEventRecord(h->ev_join[c - 1], h->side[c - 1]);
            }
        }
        launch_class<RG, RS>(h, X, fac, cv, *h->lcls[0], h->stream);
        for (int c = 1; c < nc; ++c) cudaStreamWaitEvent(h->stream, h->ev_join[c - 1], 0);
        *launches += nc;
    } else {
        for (int k = 0; k < K; ++k) {
            kern<<<S, nt, h->areas_h[k].smem_bytes, h->stream>>>(h->d_areas.p, h->T, X, nullptr, k, fac,
                                                                 cv, h->bh.p, vs);
            ++*launches;
        }
    }
}

template <class RG, class RS>
void launch_back(mase_handle *h, const State &X, const RG *fac, const RS *cv, const double *dxG,
                 int *launches) {
    const int S = h->n_snap, K = h->S.K;
    if (h->opt.schedule == MASE_BATCHED) {
        k_back<RG, RS><<<K * S, h->back_threads, h->smem_back, h->stream>>>(
            h->d_areas.p, h->T, X, h->d_inst.p, -1, fac, cv, dxG, h->bnd.n_gamma);
        ++*launches;
    } else {
        for (int k = 0; k < K; ++k) {
            const size_t sm = (size_t)h->areas_h[k].back_smem_bytes;
            k_back<RG, RS><<<S, h->back_threads, sm, h->stream>>>(h->d_areas.p, h->T, X, nullptr, k, fac,
                                                               cv, dxG, h->bnd.n_gamma);
            ++*launches;
        }
    }
}

template <class RG, class RS>
int enqueue_step(mase_handle *h, int *launches) {
    State X = make_state(h);
    cudaStream_t st = h->stream;
    const int S = h->n_snap, nt = h->threads;
    RG *fac = (RG *)h->fac.p;
    RS *cv = (RS *)h->cvec.p;
    mark(h, 0);
    State Xa = X, Xc = X, Xb = X;
    Xa.clk = h->clk.p;
    Xc.clk = h->clk.p + 2;
    Xb.clk = h->clk.p + 4;
    // local Gauss-Newton steps with the boundary held fixed (Eq. local_wls):
    // the area pass, then the interior recovery with a zero boundary step.
    // Both count towards the area stage's clock, so that the stages' spans
    // within a step stay disjoint.
    for (int q = 0; q < h->opt.inner_iters; ++q) {
        launch_local<RG, RS>(h, Xa, fac, cv, launches);
        launch_back<RG, RS>(h, Xa, fac, cv, h->dx_zero.p, launches);
    }
    if (h->opt.inner_iters > 0) {
        // the outer step alone decides convergence
        k_clear_step<<<(S + 255) / 256, 256, 0, st>>>(X);
        ++*launches;
    }
    launch_local<RG, RS>(h, Xa, fac, cv, launches);
    mark(h, 1);
    if (h->bnd.n_gamma > 0) {
        const int refine = h->opt.precision == MASE_MIXED ? h->opt.refine : 0;
        if (h->bnd_cluster)
            k_boundary_cl<RG, RS><<<2 * S, nt, h->smem_bnd_cl, st>>>(h->T, Xc, h->bnd, fac, h->bh.p,
                                                                   (RG *)h->bA.p, h->dxG.p, refine);
        else
            k_boundary<RG, RS><<<S, nt, h->smem_bnd, st>>>(h->d_areas.p, h->T, Xc, h->bnd, fac, h->bh.p,
                                                          (RG *)h->bst.p, (RG *)h->bA.p, h->dxG.p,
                                                          refine);
        ++*launches;
    }
    mark(h, 2);
    launch_back<RG, RS>(h, Xb, fac, cv, h->dxG.p, launches);
    mark(h, 3);
    return MASE_OK;
}

// Bookkeeping after a step.  Inside the solve graph it also sets the
// condition of the device-side loop; stepping from the host, the host reads
// the count of snapshots still iterating.
int enqueue_finalize(mase_handle *h, int *launches, bool in_graph) {
    State X = make_state(h);
    k_finalize<<<1, 1024, 0, h->stream>>>(X, h->iters.p, h->status.p, h->laststep.p, h->stop.p,
                                         make_ctl(h), h->loop_cond, in_graph ? 1 : 0);
    ++*launches;
    mark(h, 4);
    if (!in_graph)
        CK(cudaMemcpyAsync(h->h_n_active, h->n_active.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return MASE_OK;
}

// The Gauss-Newton loop as one graph: a while node whose body is one step
// and whose condition the bookkeeping kernel sets (snapshots still active and
// steps below max_iter); the condition starts at 1 on every launch.
template <class RG, class RS>
int build_loop_graph(mase_handle *h) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    h->graph = g;
    CK(cudaGraphConditionalHandleCreate(&h->loop_cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h->loop_cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    int per_step = 0;
    int rc = enqueue_step<RG, RS>(h, &per_step);
    int rc2 = rc == MASE_OK ? enqueue_finalize(h, &per_step, true) : rc;
    cudaGraph_t captured = nullptr;
    cudaError_t ce = cudaStreamEndCapture(h->stream, &captured);
    if (rc != MASE_OK) return rc;
    if (rc2 != MASE_OK) return rc2;
    CK(ce);
    h->graph_launches = per_step;
    CK(cudaGraphInstantiate(&h->graph_exec, g, 0));
    return MASE_OK;
}

int enqueue_objective(mase_handle *h, int *launches) {
    mase_internal::launch_objective(h, h->xV.p, h->xT.p, h->J.p, launches);
    return MASE_OK;
}

template <class RG, class RS>
int build(mase_handle *h) {
    mase::Setup &S = h->S;
    cudaStream_t st = h->stream;
    const int K = S.K, nS = h->n_snap;
    HostTables &H = h->H;
    h->areas_h.resize(K);
    size_t max_local = 0, max_back = 0;
    long long fac_off = 0, c_off = 0, bh_off = 0;
    int in_smem_count = 0;
    long long factor_nnz = 0, local_flops = 0, gup = 0;
    int max_vars = 0, max_nb = 0;
    for (int k = 0; k < K; ++k) {
        const mase::AreaSetup &A = S.areas[k];
        AreaDev d{};
        d.F = append_fac(H, A.F);
        d.nb_int = A.nb_int;
        d.nb_loc = A.nb_loc;
        d.n_own = A.n_own;
        d.n_ends = A.n_ends;
        d.n_slots = A.n_slots;
        d.n_items = A.n_items;
        d.bus_base = (int)H.locbus.size();
        app(H.locbus, A.locbus);
        app(H.qvarV, A.qvarV);
        app(H.qvarT, A.qvarT);
        d.own_base = (int)H.own_q.size();
        app(H.own_q, A.own_q);
        app(H.own_gvv, A.own_gvv);
        d.own1_base = (int)H.own_ebeg.size();
        app(H.own_ebeg, A.own_ebeg);
        d.end_base = (int)H.end_qi.size();
        app(H.end_qi, A.end_qi);
        app(H.end_qj, A.end_qj);
        app(H.end_own, A.end_own);
        app(H.end_var, A.end_var);
        app(H.end_gpos, A.end_gpos);
        app(H.end_g, A.end_g);
        app(H.end_b, A.end_b);
        app(H.end_bh, A.end_bh);
        d.item_base = (int)(H.item_pos.size() / 4);
        app(H.item_pos, A.item_pos);
        app(H.item_rec, A.item_rec);
        d.ebnd_base = (int)H.ebnd.size();
        app(H.ebnd, A.ebnd);
        d.zrow_base = S.zrow_base[k];
        // dynamic shared memory layout
        const int nv = A.n_int + A.n_bnd;
        const mase::SmemLayout lay =
            mase::area_smem_layout(nv, A.nb_loc, A.n_ends, A.n_own, sizeof(RG), sizeof(RS));
        d.off_g = (int)lay.off_g;
        d.off_y = (int)lay.off_y;
        d.off_bus = (int)lay.off_bus;
        d.off_end = (int)lay.off_end;
        d.off_inj = (int)lay.off_inj;
        d.off_self = (int)lay.off_self;
        d.off_st = (int)lay.off_st;
        const size_t o = lay.vector_bytes;
        const size_t with_st = o + (size_t)A.F.store_total * sizeof(RG);
        const size_t ctr_bytes = ((2 * (size_t)A.F.nsn() + 1) * sizeof(int) + 15) & ~size_t(15);
        d.vec_global = 0;
        d.vec_stride = 0;
        d.vec_base = 0;
        if (with_st <= (size_t)h->smem_limit) {
            d.in_smem = 1;
            d.smem_bytes = (int)with_st;
            ++in_smem_count;
        } else if (o <= (size_t)h->smem_limit) {
            d.in_smem = 0;
            d.smem_bytes = (int)o;
        } else {
            // vectors and factor in global memory, dataflow counters on chip
            if (ctr_bytes > (size_t)h->smem_limit)
                return set_err(MASE_EINVAL, "area " + std::to_string(k) + " too large: task counters exceed shared memory");
            d.in_smem = 0;
            d.vec_global = 1;
            d.smem_bytes = (int)ctr_bytes;
            d.vec_stride = (int)((o + 255) & ~size_t(255));
            d.vec_base = h->vscratch_bytes;
            h->vscratch_bytes += (long long)d.vec_stride * nS;
            h->vec_global = 1;
        }
        // the factorisation's task counters reuse the bus-value region
        if (!d.vec_global && ctr_bytes > 3 * (size_t)A.nb_loc * sizeof(double))
            return set_err(MASE_EINVAL, "area " + std::to_string(k) + ": task counters do not fit");
        max_local = std::max(max_local, (size_t)d.smem_bytes);
        d.back_smem_bytes = (int)(((size_t)nv * sizeof(RS) + 15) & ~size_t(15));
        d.obj_off_end = (int)((3 * (size_t)A.nb_loc * sizeof(double) + 15) & ~size_t(15));
        d.obj_smem_bytes = d.obj_off_end + 16 * A.n_ends;
        if (!d.vec_global) h->smem_obj = std::max(h->smem_obj, (size_t)d.obj_smem_bytes);
        max_back = std::max(max_back, (size_t)d.back_smem_bytes);
        d.fac_base = fac_off;
        // instance bases stay 16-byte aligned
        d.fac_stride = (A.F.store_total + 3) & ~3;
        fac_off += (long long)d.fac_stride * nS;
        d.c_base = c_off;
        c_off += (long long)A.n_int * nS;
        d.bh_base = bh_off;
        bh_off += (long long)A.n_bnd * nS;
        h->areas_h[k] = d;
        factor_nnz += A.F.store_total;
        local_flops += A.F.flops;
        gup += A.g_updates;
        h->info.n_supernodes += A.F.nsn();
        h->info.n_units += (int64_t)A.F.unit_sn.size();
        h->info.max_levels = std::max(h->info.max_levels, A.F.nlev());
        h->info.max_area_store = std::max(h->info.max_area_store, A.F.store_total);
        max_vars = std::max(max_vars, nv);
        max_nb = std::max(max_nb, A.n_bnd);
        h->info.coord_S_elems += (int64_t)A.n_bnd * (A.n_bnd + 1) / 2;
        h->info.coord_b_elems += A.n_bnd;
    }
    h->fac_elems = fac_off;
    h->c_elems = c_off;
    h->bh_elems = bh_off;
    h->smem_local = max_local;
    h->smem_back = max_back;
    // boundary system
    const mase::BoundarySetup &B = S.B;
    BndDev &bd = h->bnd;
    bd.F = append_fac(H, B.F);
    bd.n_gamma = B.n_gamma;
    bd.stride = B.F.store_total;
    {
        // vectors first, then as much of the top of the boundary factor as fits
        const size_t vec0 = (((size_t)B.n_gamma * (3 * sizeof(double) + sizeof(RS))) + 15) & ~size_t(15);
        // task counters of the dataflow factorisation
        const size_t vec = vec0 + ((((size_t)2 * B.F.nsn() + 1) * sizeof(int) + 15) & ~size_t(15));
        bd.smem_off_ctr = (int)vec0;
        if (vec > (size_t)h->smem_limit)
            return set_err(MASE_EINVAL, "boundary system too large for shared-memory vectors");
        const long long room = ((long long)h->smem_limit - (long long)vec) / (long long)sizeof(RG);
        int split = B.F.store_total;
        for (int sn = 0; sn < B.F.nsn(); ++sn)
            if ((long long)B.F.store_total - B.F.sn_off[sn] <= room) {
                split = B.F.sn_off[sn];
                break;
            }
        bd.split = split;
        bd.smem_off_st = (int)vec;
        h->smem_bnd = vec + (size_t)(B.F.store_total - split) * sizeof(RG);
        // MIXED: a 2-block cluster holds the rest of the factor in its second
        // block's shared memory when it fits
        bd.split_cl = split;
        h->bnd_cluster = 0;
        if (h->opt.precision == MASE_MIXED && (size_t)split * sizeof(RG) <= (size_t)h->smem_limit &&
            2 * (size_t)nS <= 65535) {
            h->bnd_cluster = 1;
            h->smem_bnd_cl = std::max(h->smem_bnd, (size_t)split * sizeof(RG));
        }
    }
    // instance list: areas by descending work, snapshots innermost
    std::vector<int> ord(K);
    for (int k = 0; k < K; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return S.areas[a].work > S.areas[b].work; });
    h->inst_h.clear();
    for (int k : ord)
        for (int s = 0; s < nS; ++s) h->inst_h.push_back(make_int2(k, s));
    // default launch configuration: one class holding every area
    h->area_order = ord;
    h->lcls.clear();
    h->lcls.emplace_back(new LocalClass());
    h->lcls[0]->threads = h->threads;
    h->lcls[0]->smem = h->smem_local;
    h->lcls[0]->n_areas = K;
    h->lcls[0]->inst_h = h->inst_h;
    h->back_threads = kBackThreads;
    // uploads
#define UP(buf, vec) CK(h->buf.upload(H.vec, st))
    UP(t_sn_c0, sn_c0); UP(t_sn_w, sn_w); UP(t_sn_nr, sn_nr); UP(t_sn_off, sn_off);
    UP(t_sn_order, sn_order);
    UP(t_lev_off, lev_off); UP(t_rows, rows);
    UP(t_rel, rel); UP(t_locbus, locbus); UP(t_qvarV, qvarV);
    UP(t_qvarT, qvarT); UP(t_own_q, own_q); UP(t_own_gvv, own_gvv); UP(t_own_ebeg, own_ebeg);
    UP(t_end_qi, end_qi); UP(t_end_qj, end_qj); UP(t_end_own, end_own);
    UP(t_end_var, end_var); UP(t_end_gpos, end_gpos); UP(t_end_g, end_g); UP(t_end_b, end_b);
    UP(t_end_bh, end_bh);
    UP(t_item_pos, item_pos); UP(t_ebnd, ebnd);
#undef UP
    CK(h->b_asm_beg.upload(B.asm_beg, st));
    CK(h->b_asm_area.upload(B.asm_area, st));
    CK(h->b_asm_off.upload(B.asm_off, st));
    CK(h->b_rhs_beg.upload(B.rhs_beg, st));
    CK(h->b_rhs_area.upload(B.rhs_area, st));
    CK(h->b_rhs_lv.upload(B.rhs_lv, st));
    CK(h->b_bvar_ibus.upload(B.bvar_ibus, st));
    CK(h->b_bvar_isT.upload(B.bvar_isT, st));
    {
        // absolute gather sources: instance base + offset, plus the per-snapshot stride
        std::vector<long long> aabs(B.asm_area.size()), rabs(B.rhs_area.size());
        std::vector<int> astr(B.asm_area.size()), rstr(B.rhs_area.size());
        for (size_t i = 0; i < B.asm_area.size(); ++i) {
            const AreaDev &A = h->areas_h[B.asm_area[i]];
            aabs[i] = A.fac_base + B.asm_off[i];
            astr[i] = A.fac_stride;
        }
        for (size_t i = 0; i < B.rhs_area.size(); ++i) {
            const AreaDev &A = h->areas_h[B.rhs_area[i]];
            rabs[i] = A.bh_base + B.rhs_lv[i];
            rstr[i] = A.F.n_bnd;
        }
        CK(h->b_asm_abs.upload(aabs, st));
        CK(h->b_asm_str.upload(astr, st));
        CK(h->b_rhs_abs.upload(rabs, st));
        CK(h->b_rhs_str.upload(rstr, st));
        bd.asm_abs = h->b_asm_abs.p;
        bd.asm_str = h->b_asm_str.p;
        bd.rhs_abs = h->b_rhs_abs.p;
        bd.rhs_str = h->b_rhs_str.p;
    }
    bd.asm_beg = h->b_asm_beg.p;
    bd.asm_area = h->b_asm_area.p;
    bd.asm_off = h->b_asm_off.p;
    bd.rhs_beg = h->b_rhs_beg.p;
    bd.rhs_area = h->b_rhs_area.p;
    bd.rhs_lv = h->b_rhs_lv.p;
    bd.bvar_ibus = h->b_bvar_ibus.p;
    bd.bvar_isT = h->b_bvar_isT.p;
    std::vector<AreaDev> ah = h->areas_h;
    CK(h->d_areas.upload(ah, st));
    CK(h->d_inst.upload(h->inst_h, st));
    CK(h->lcls[0]->inst.upload(h->lcls[0]->inst_h, st));
    Tables &T = h->T;
    // a dependency wait gives up after this many unsatisfied polls (~0.2 s by default)
    T.wait_polls = h->opt.wait_polls > 0 ? h->opt.wait_polls : (1 << 22);
    T.mma_min_w = h->opt.precision == MASE_MIXED ? h->opt.tensor_units : 0;
    T.sn_c0 = h->t_sn_c0.p; T.sn_w = h->t_sn_w.p; T.sn_nr = h->t_sn_nr.p; T.sn_off = h->t_sn_off.p;
    T.sn_order = h->t_sn_order.p;
    T.lev_off = h->t_lev_off.p; T.rows = h->t_rows.p;
    T.rel = h->t_rel.p;
    T.locbus = h->t_locbus.p; T.qvarV = h->t_qvarV.p; T.qvarT = h->t_qvarT.p;
    T.own_q = h->t_own_q.p; T.own_gvv = h->t_own_gvv.p; T.own_ebeg = h->t_own_ebeg.p;
    T.end_qi = h->t_end_qi.p; T.end_qj = h->t_end_qj.p;
    T.end_own = h->t_end_own.p; T.end_var = h->t_end_var.p; T.end_gpos = h->t_end_gpos.p;
    T.end_g = h->t_end_g.p; T.end_b = h->t_end_b.p; T.end_bh = h->t_end_bh.p;
    T.item_pos = h->t_item_pos.p;
    T.ebnd = h->t_ebnd.p;
    CK(h->t_tasks.upload(H.tasks.empty() ? std::vector<int>(16, 0) : H.tasks, st));
    T.task_rec = reinterpret_cast<const int4 *>(h->t_tasks.p);
    CK(h->t_lev_tasks.upload(H.lev_tasks, st));
    T.lev_tasks = h->t_lev_tasks.p;
    CK(h->t_item_rec.upload(H.item_rec, st));
    T.item_rec = reinterpret_cast<const int4 *>(h->t_item_rec.p);
    CK(h->t_chunk_rec.upload(H.chunk_rec.empty() ? std::vector<int>(8, 0) : H.chunk_rec, st));
    CK(h->t_lev_chunks.upload(H.lev_chunks, st));
    T.chunk_rec = reinterpret_cast<const int4 *>(h->t_chunk_rec.p);
    T.lev_chunks = h->t_lev_chunks.p;
    // work buffers
    CK(h->fac.alloc((size_t)h->fac_elems * sizeof(RG)));
    CK(h->vscratch.alloc((size_t)std::max<long long>(16, h->vscratch_bytes)));
    CK(h->cvec.alloc((size_t)std::max<long long>(1, h->c_elems) * sizeof(RS)));
    CK(h->bh.alloc((size_t)std::max<long long>(1, h->bh_elems)));
    CK(h->bst.alloc((size_t)std::max(1, B.F.store_total) * nS * sizeof(RG)));
    CK(h->bA.alloc((size_t)std::max(1, B.F.store_total) * nS * sizeof(RG)));
    CK(h->dxG.alloc((size_t)std::max(1, B.n_gamma) * nS));
    CK(h->dx_zero.alloc((size_t)std::max(1, B.n_gamma) * nS));
    CK(cudaMemsetAsync(h->dx_zero.p, 0, (size_t)std::max(1, B.n_gamma) * nS * sizeof(double), st));
    setup_attrs<RG, RS>(h);
    // info
    mase_info &I = h->info;
    I.n_bus = S.N;
    I.n_branch = S.L;
    I.n_area = S.K;
    I.n_snap = nS;
    I.n_meas = S.m;
    I.n_state = 2 * S.N - 1;
    I.n_boundary_bus = S.n_boundary_bus;
    I.n_gamma = B.n_gamma;
    I.max_area_vars = max_vars;
    I.max_area_nb = max_nb;
    I.factor_nnz = factor_nnz;
    I.local_flops = local_flops;
    I.boundary_flops = B.F.flops;
    I.g_updates = gup;
    I.smem_bytes_max = (int)max_local;
    I.areas_in_smem = in_smem_count;
    I.boundary_store = B.F.store_total;
    I.boundary_levels = B.F.nlev();
    return MASE_OK;
}

// ---------------------------------------------------------------------------
// autotuner: the launch configuration measured on the device at create
// ---------------------------------------------------------------------------
// Best of `reps` timings (CUDA events on the library's stream) after one
// untimed run.
template <class F>
float time_min(mase_handle *h, F fn, int reps) {
    fn();
    float best = 1e30f;
    for (int i = 0; i < reps; ++i) {
        cudaEventRecord(h->ev_solve[0], h->stream);
        fn();
        cudaEventRecord(h->ev_solve[1], h->stream);
        cudaEventSynchronize(h->ev_solve[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_solve[0], h->ev_solve[1]);
        best = std::min(best, ms);
    }
    return best;
}

// The tuning problem is the network at the flat start with z = h(x_flat) in
// every snapshot: the same sparsity, task lists and instance counts as any
// batch of real measurements, so the timings carry over, and no measurement
// of the caller is needed.  Candidates:
//  * area-to-block packing: areas grouped into classes by how many of their
//    blocks fit on one SM by shared memory (1, 2, 3+), each class launched
//    on its own stream with its own dynamic shared memory; per class the
//    block size is chosen among those whose registers still allow that many
//    blocks per SM; the split is kept only if it beats one launch for all;
//  * block size of the back-substitution;
//  * coordinator on 2-block clusters or on one block (factor top on chip).
template <class RG, class RS>
int autotune(mase_handle *h) {
    mase_info &I = h->info;
    I.local_classes = 1;
    I.class_areas[0] = h->S.K;
    I.class_threads[0] = h->threads;
    I.class_smem[0] = (int)h->smem_local;
    I.back_threads = h->back_threads;
    I.coord_cluster = h->bnd_cluster;
    if (h->opt.schedule != MASE_BATCHED || !h->opt.autotune) return MASE_OK;
    cudaStream_t st = h->stream;
    const int K = h->S.K, nS = h->n_snap, M = h->S.m, N = h->S.N;
    for (int s = 0; s < nS; ++s)
        CK(cudaMemcpyAsync(h->z_int.p + (size_t)s * M, h->h_flat.p, (size_t)M * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
    State X = make_state(h);
    X.mask = nullptr;
    k_state_in<<<1024, 256, 0, st>>>(nullptr, h->xV.p, h->xT.p, h->bus_of_ibus.p, N, nS, 1);
    k_reset<<<(nS + 255) / 256, 256, 0, st>>>(X, h->iters.p, h->status.p, h->laststep.p, make_ctl(h));
    CK(cudaGetLastError());
    RG *fac = (RG *)h->fac.p;
    RS *cv = (RS *)h->cvec.p;
    int nl = 0;
    auto run_local = [&]() { launch_local<RG, RS>(h, X, fac, cv, &nl); };
    const float t_single = time_min(h, run_local, 3);
    // classes by blocks per SM that fit by shared memory, in descending-work order
    std::vector<std::vector<int>> by_cap(4);
    for (int k : h->area_order) {
        const size_t need = (size_t)h->areas_h[k].smem_bytes + 1024;
        const int cap = (int)std::min<size_t>(3, std::max<size_t>(1, kSmemPerSM / need));
        by_cap[cap].push_back(k);
    }
    std::vector<std::unique_ptr<LocalClass>> single;
    single.swap(h->lcls);
    std::vector<int> caps;
    for (int cap = 1; cap <= 3; ++cap) {
        if (by_cap[cap].empty()) continue;
        caps.push_back(cap);
        std::unique_ptr<LocalClass> c(new LocalClass());
        c->n_areas = (int)by_cap[cap].size();
        for (int k : by_cap[cap]) {
            c->smem = std::max(c->smem, (size_t)h->areas_h[k].smem_bytes);
            for (int s = 0; s < nS; ++s) c->inst_h.push_back(make_int2(k, s));
        }
        CK(c->inst.upload(c->inst_h, st));
        c->threads = h->threads;
        h->lcls.push_back(std::move(c));
    }
    float t_split = 1e30f;
    if (h->lcls.size() > 1 || (caps.size() == 1 && caps[0] > 1)) {
        // block size per class, the class timed alone
        for (size_t ci = 0; ci < h->lcls.size(); ++ci) {
            LocalClass &c = *h->lcls[ci];
            const int cap = caps[ci];
            int best_t = h->threads;
            float best = 1e30f;
            for (int t : {512, 256, 160}) {
                if (t > h->threads || (t != h->threads && (long long)t * cap > 512)) continue;
                c.threads = t;
                const float ms = time_min(h, [&]() { launch_class<RG, RS>(h, X, fac, cv, c, st); }, 3);
                if (ms < best) {
                    best = ms;
                    best_t = t;
                }
            }
            c.threads = best_t;
        }
        t_split = time_min(h, run_local, 3);
    }
    CK(cudaGetLastError());
    if (!(t_split < 0.99f * t_single)) {
        h->lcls.swap(single);   // one launch for every area stays
        t_split = t_single;
    }
    // back-substitution block size
    launch_local<RG, RS>(h, X, fac, cv, &nl);
    {
        int best_t = h->back_threads;
        float best = 1e30f;
        for (int t : {256, 128}) {
            h->back_threads = t;
            const float ms = time_min(h, [&]() { launch_back<RG, RS>(h, X, fac, cv, h->dx_zero.p, &nl); }, 3);
            if (ms < best) {
                best = ms;
                best_t = t;
            }
        }
        h->back_threads = best_t;
    }
    // coordinator form
    if (h->bnd.n_gamma > 0 && h->bnd_cluster) {
        const int refine = h->opt.precision == MASE_MIXED ? h->opt.refine : 0;
        const int nt = h->threads;
        const float t_cl = time_min(h, [&]() {
            k_boundary_cl<RG, RS><<<2 * nS, nt, h->smem_bnd_cl, st>>>(h->T, X, h->bnd, fac, h->bh.p,
                                                                    (RG *)h->bA.p, h->dxG.p, refine);
        }, 3);
        const float t_one = time_min(h, [&]() {
            k_boundary<RG, RS><<<nS, nt, h->smem_bnd, st>>>(h->d_areas.p, h->T, X, h->bnd, fac, h->bh.p,
                                                           (RG *)h->bst.p, (RG *)h->bA.p, h->dxG.p, refine);
        }, 3);
        h->bnd_cluster = t_cl <= t_one ? 1 : 0;
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    I.tuned = 1;
    I.local_classes = (int)h->lcls.size();
    for (int c = 0; c < 4; ++c) I.class_areas[c] = I.class_threads[c] = I.class_smem[c] = 0;
    for (size_t c = 0; c < h->lcls.size() && c < 4; ++c) {
        I.class_areas[c] = h->lcls[c]->n_areas;
        I.class_threads[c] = h->lcls[c]->threads;
        I.class_smem[c] = (int)h->lcls[c]->smem;
    }
    I.back_threads = h->back_threads;
    I.coord_cluster = h->bnd_cluster;
    I.tune_local_ms[0] = t_single;
    I.tune_local_ms[1] = t_split;
    return MASE_OK;
}

int upload_measurements(mase_handle *h, const mase_measurements *meas) {
    cudaStream_t st = h->stream;
    const int M = h->S.m, nS = h->n_snap;
    const size_t n = (size_t)M * nS;
    if (meas->z) {
        const double *src = meas->z;
        if (!is_device_ptr(meas->z)) {
            CK(cudaMemcpyAsync(h->z_stage.p, meas->z, n * sizeof(double), cudaMemcpyHostToDevice, st));
            src = h->z_stage.p;
        }
        k_gather_rows<<<1024, 256, 0, st>>>(src, h->z_int.p, h->zperm.p, M, nS);
        CK(cudaGetLastError());
        h->has_z = true;
    }
    if (meas->mask) {
        if (!h->has_mask && h->graph_exec) {
            // the captured loop reads the mask pointer it was captured with
            cudaGraphExecDestroy(h->graph_exec);
            cudaGraphDestroy(h->graph);
            h->graph_exec = nullptr;
            h->graph = nullptr;
        }
        if (!h->mask_int.p) {
            CK(h->mask_int.alloc(n));
            CK(h->mask_stage.alloc(n));
        }
        const uint8_t *src = meas->mask;
        if (!is_device_ptr(meas->mask)) {
            CK(cudaMemcpyAsync(h->mask_stage.p, meas->mask, n, cudaMemcpyHostToDevice, st));
            src = h->mask_stage.p;
        }
        k_gather_mask<<<1024, 256, 0, st>>>(src, h->mask_int.p, h->zperm.p, M, nS);
        CK(cudaGetLastError());
        h->has_mask = true;
    }
    CK(cudaStreamSynchronize(st));
    return MASE_OK;
}

template <class RG, class RS>
int solve_impl(mase_handle *h, const double *x0, double tol, int max_iter, double *x_out,
               mase_stats *stats) {
    cudaStream_t st = h->stream;
    const int N = h->S.N, nS = h->n_snap;
    int launches = 0;
    State X = make_state(h);
    // events: solve start, learned start begin/end, loop begin/end, solve end
    cudaEvent_t *ev = h->ev_solve;
    CK(cudaEventRecord(ev[0], st));
    k_reset<<<(nS + 255) / 256, 256, 0, st>>>(X, h->iters.p, h->status.p, h->laststep.p, make_ctl(h));
    ++launches;
    if (x0) {
        const double *src = x0;
        if (!is_device_ptr(x0)) {
            CK(cudaMemcpyAsync(h->xbuf.p, x0, (size_t)2 * N * nS * sizeof(double),
                               cudaMemcpyHostToDevice, st));
            src = h->xbuf.p;
        }
        k_state_in<<<1024, 256, 0, st>>>(src, h->xV.p, h->xT.p, h->bus_of_ibus.p, N, nS, 0);
    } else {
        k_state_in<<<1024, 256, 0, st>>>(nullptr, h->xV.p, h->xT.p, h->bus_of_ibus.p, N, nS, 1);
    }
    ++launches;
    CK(cudaGetLastError());
    CK(cudaEventRecord(ev[1], st));
    const bool learned = !x0 && h->start_mode == MASE_START_LEARNED;
    if (learned) {
        int rc = mase_internal::learned_start(h, &launches);
        if (rc != MASE_OK) return rc;
    }
    CK(cudaEventRecord(ev[2], st));
    // the stop rule goes through pinned host memory: the previous solve has
    // finished with it (every solve ends with a stream synchronisation)
    h->h_stop->tol = tol;
    h->h_stop->max_iter = max_iter;
    CK(cudaMemcpyAsync(h->stop.p, h->h_stop, sizeof(StopRule), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ev[3], st));
    const bool device_loop = h->opt.use_graph && !h->opt.profile;
    double ev_acc[4] = {0, 0, 0, 0};
    auto run_loop = [&]() -> int {
        if (device_loop) {
            if (!h->graph_exec) {
                int rc = build_loop_graph<RG, RS>(h);
                if (rc != MASE_OK) return rc;
            }
            CK(cudaGraphLaunch(h->graph_exec, st));
            return MASE_OK;
        }
        for (int it = 0; it < max_iter; ++it) {
            int rc = enqueue_step<RG, RS>(h, &launches);
            if (rc != MASE_OK) return rc;
            rc = enqueue_finalize(h, &launches, false);
            if (rc != MASE_OK) return rc;
            CK(cudaStreamSynchronize(st));
            CK(cudaGetLastError());
            if (h->opt.profile) {
                for (int i = 0; i < 4; ++i) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, h->ev_stage[i], h->ev_stage[i + 1]));
                    ev_acc[i] += ms;
                }
            }
            if (*h->h_n_active == 0) break;
        }
        return MASE_OK;
    };
    std::vector<int> iters(nS), status(nS), picked(nS, 0);
    std::vector<double> J(nS), last(nS);
    double acc[4] = {0, 0, 0, 0};
    int gemm_err = 0;
    int steps = 0;
    // objective at the final states, the states out and the per-snapshot results
    auto finish = [&]() -> int {
        CK(cudaEventRecord(ev[4], st));
        int rc = enqueue_objective(h, &launches);
        if (rc != MASE_OK) return rc;
        if (x_out) {
            if (is_device_ptr(x_out)) {
                k_state_out<<<1024, 256, 0, st>>>(x_out, h->xV.p, h->xT.p, h->bus_of_ibus.p, N, nS);
            } else {
                k_state_out<<<1024, 256, 0, st>>>(h->xbuf.p, h->xV.p, h->xT.p, h->bus_of_ibus.p, N, nS);
                CK(cudaMemcpyAsync(x_out, h->xbuf.p, (size_t)2 * N * nS * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
            }
            ++launches;
        }
        int steps_now = 0;
        CK(cudaMemcpyAsync(iters.data(), h->iters.p, nS * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(status.data(), h->status.p, nS * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(J.data(), h->J.p, nS * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(last.data(), h->laststep.p, nS * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(acc, h->clk_acc.p, sizeof(acc), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&steps_now, h->steps_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (learned) {
            CK(cudaMemcpyAsync(picked.data(), mase_internal::learned_picked(h), nS * sizeof(int),
                               cudaMemcpyDeviceToHost, st));
            if (int *ge = mase_internal::learned_gemm_err(h))
                CK(cudaMemcpyAsync(&gemm_err, ge, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        CK(cudaEventRecord(ev[5], st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        steps += steps_now;
        if (device_loop) launches += h->graph_launches * steps_now;
        return MASE_OK;
    };
    int n_restarted = 0;
    int rc = run_loop();
    if (rc != MASE_OK) return rc;
    rc = finish();
    if (rc != MASE_OK) return rc;
    if (gemm_err) {
        CK(cudaMemsetAsync(mase_internal::learned_gemm_err(h), 0, sizeof(int), st));
        return set_err(MASE_EDEVICE, "a tensor-core GEMM of the learned start gave up a bounded wait");
    }
    // flat-start fallback: a snapshot that started from the networks'
    // proposal and whose factor broke down (non-positive pivot or non-finite
    // step) is solved again from the flat start; its iteration count keeps
    // the steps spent on the failed attempt
    if (learned) {
        std::vector<int> again(nS, 0), spent(nS, 0);
        int n_again = 0;
        for (int s = 0; s < nS; ++s)
            if (picked[s] && (status[s] == MASE_SNAP_NOT_SPD || status[s] == MASE_SNAP_NONFINITE)) {
                again[s] = 1;
                spent[s] = iters[s];
                ++n_again;
            }
        if (n_again) {
            if (!h->restart.p) CK(h->restart.alloc(nS));
            CK(cudaMemcpyAsync(h->restart.p, again.data(), nS * sizeof(int), cudaMemcpyHostToDevice, st));
            k_restart<<<1024, 256, 0, st>>>(X, h->iters.p, h->status.p, h->laststep.p, h->restart.p,
                                            make_ctl(h));
            ++launches;
            CK(cudaGetLastError());
            rc = run_loop();
            if (rc != MASE_OK) return rc;
            rc = finish();
            if (rc != MASE_OK) return rc;
            for (int s = 0; s < nS; ++s) iters[s] += spent[s];
        }
        n_restarted = n_again;
    }
    if (h->opt.profile)
        for (int i = 0; i < 4; ++i) acc[i] = ev_acc[i];
    // the batch's code is that of its worst snapshot, whatever their order:
    // a device wait that gave up, then a non-positive pivot, then a
    // non-finite step, then the iteration cap
    int worst = 0;
    for (int s = 0; s < nS; ++s) {
        const int st = status[s];
        const int rank = st == MASE_SNAP_DEVICE ? 4 : st == MASE_SNAP_NOT_SPD ? 3
                       : st == MASE_SNAP_NONFINITE ? 2 : st == MASE_SNAP_MAX_ITER ? 1 : 0;
        worst = std::max(worst, rank);
    }
    static const int kRetOfRank[5] = {MASE_OK, MASE_NOT_CONVERGED, MASE_ENONFINITE, MASE_EUNOBSERVABLE,
                                      MASE_EDEVICE};
    const int ret = kRetOfRank[worst];
    if (stats) {
        for (int s = 0; s < nS; ++s) {
            if (stats->iters) stats->iters[s] = iters[s];
            if (stats->status) stats->status[s] = status[s];
            if (stats->J) stats->J[s] = J[s];
            if (stats->max_step) stats->max_step[s] = last[s];
        }
        stats->total_launches = launches;
        stats->steps = steps;
        stats->restarted = n_restarted;
        float t_all = 0.f, t_pre = 0.f, t_ws = 0.f, t_stop = 0.f, t_loop = 0.f, t_post = 0.f;
        CK(cudaEventElapsedTime(&t_all, ev[0], ev[5]));
        CK(cudaEventElapsedTime(&t_pre, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&t_ws, ev[1], ev[2]));
        CK(cudaEventElapsedTime(&t_stop, ev[2], ev[3]));
        CK(cudaEventElapsedTime(&t_loop, ev[3], ev[4]));
        CK(cudaEventElapsedTime(&t_post, ev[4], ev[5]));
        for (int i = 0; i < 4; ++i) stats->stage_ms[i] = acc[i];
        stats->stage_ms[4] = t_ws;
        stats->stage_ms[5] = (double)t_pre + t_stop + t_post;
        // what the loop spent outside its stages' kernels: launch gaps and,
        // when stepping from the host, the round trip of every step
        stats->stage_ms[6] = (double)t_loop - (acc[0] + acc[1] + acc[2] + acc[3]);
        stats->solve_ms = t_all;
    }
    if (ret == MASE_EUNOBSERVABLE) set_err(ret, "non-positive pivot in an area or boundary factor");
    if (ret == MASE_ENONFINITE) set_err(ret, "non-finite step");
    if (ret == MASE_EDEVICE) set_err(ret, "a bounded device-side wait gave up");
    return ret;
}

}  // namespace

extern "C" {

void mase_default_options(mase_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = MASE_MIXED;
    o->schedule = MASE_BATCHED;
    o->use_graph = 1;
    o->refine = 1;
    o->threads = 0;
    o->device = 0;
    o->stream = nullptr;
    o->profile = 0;
    o->wait_polls = 0;
    o->inner_iters = 0;
    o->autotune = 1;
    o->tensor_units = kDefaultTensorUnits;
}

const char *mase_status_str(int code) {
    switch (code) {
        case MASE_OK: return "MASE_OK";
        case MASE_NOT_CONVERGED: return "MASE_NOT_CONVERGED";
        case MASE_EINVAL: return "MASE_EINVAL";
        case MASE_EUNOBSERVABLE: return "MASE_EUNOBSERVABLE";
        case MASE_ENONFINITE: return "MASE_ENONFINITE";
        case MASE_EDEVICE: return "MASE_EDEVICE";
        case MASE_ENOTREADY: return "MASE_ENOTREADY";
        default: return "MASE_UNKNOWN";
    }
}

const char *mase_last_error(void) { return g_last_error.c_str(); }

int mase_create(const mase_network *net, const mase_partition *part, const mase_measurements *meas,
                const mase_options *opt, mase_handle **out) {
    if (!net || !part || !meas || !out) return set_err(MASE_EINVAL, "null argument");
    if (meas->n_snap < 1) return set_err(MASE_EINVAL, "n_snap must be >= 1");
    if (!meas->sigma) return set_err(MASE_EINVAL, "sigma is required");
    std::unique_ptr<mase_handle> h(new mase_handle());
    if (opt) h->opt = *opt;
    else mase_default_options(&h->opt);
    if (h->opt.precision != MASE_FP64 && h->opt.precision != MASE_MIXED)
        return set_err(MASE_EINVAL, "bad precision");
    if (h->opt.schedule != MASE_PER_AREA && h->opt.schedule != MASE_BATCHED)
        return set_err(MASE_EINVAL, "bad schedule");
    if (h->opt.refine < 0 || h->opt.refine > 8) return set_err(MASE_EINVAL, "bad refine count");
    if (h->opt.inner_iters < 0 || h->opt.inner_iters > 8)
        return set_err(MASE_EINVAL, "bad inner iteration count");
    if (h->opt.wait_polls < 0) return set_err(MASE_EINVAL, "bad wait_polls");
    if (h->opt.tensor_units == -1) h->opt.tensor_units = kDefaultTensorUnits;
    if (h->opt.tensor_units < 0 || h->opt.tensor_units > 255)
        return set_err(MASE_EINVAL, "tensor_units must be -1 or 0..255");
    int threads = h->opt.threads ? h->opt.threads : 512;
    if (threads < 64 || threads > 512 || threads % 32) return set_err(MASE_EINVAL, "bad threads");
    h->threads = threads;
    mase::NetIn ni{net->n_bus, net->n_branch, net->slack_bus, net->from_bus, net->to_bus,
                   net->r, net->x, net->b_charge};
    {
        int optin0 = 0;
        CK(cudaDeviceGetAttribute(&optin0, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->opt.device));
        h->smem_limit = optin0 - 1024;
    }
    if (!mase::build_setup(ni, part->n_area, part->area_of_bus, h->S, h->smem_limit))
        return set_err(MASE_EINVAL, h->S.error);
    const int M = h->S.m;
    for (int i = 0; i < M; ++i)
        if (!(meas->sigma[i] > 0.0) || !std::isfinite(meas->sigma[i]))
            return set_err(MASE_EINVAL, "sigma must be positive and finite");
    CK(cudaSetDevice(h->opt.device));
    h->user_stream = (cudaStream_t)h->opt.stream;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    for (auto &e : h->ev_solve) CK(cudaEventCreate(&e));
    for (auto &e : h->ev_stage) CK(cudaEventCreate(&e));
    for (auto &q : h->side) CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    for (auto &e : h->ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    {
        int rc0 = join_in(h.get());
        if (rc0 != MASE_OK) return rc0;
    }
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->opt.device));
    h->smem_limit = optin - 1024;
    h->n_snap = meas->n_snap;
    const int N = h->S.N, nS = h->n_snap;
    int rc = h->opt.precision == MASE_MIXED ? build<float, float>(h.get())
                                            : build<double, double>(h.get());
    if (rc != MASE_OK) return rc;
    cudaStream_t st = h->stream;
    // state, measurement and bookkeeping buffers
    CK(h->xV.alloc((size_t)N * nS));
    CK(h->xT.alloc((size_t)N * nS));
    CK(h->xbuf.alloc((size_t)2 * N * nS));
    CK(h->z_int.alloc((size_t)M * nS));
    CK(h->z_stage.alloc((size_t)M * nS));
    std::vector<double> Wh(M);
    for (int i = 0; i < M; ++i) {
        const double sg = meas->sigma[h->S.zperm[i]];
        Wh[i] = 1.0 / (sg * sg);
    }
    CK(h->W.upload(Wh, st));
    CK(h->zperm.upload(h->S.zperm, st));
    CK(h->bus_of_ibus.upload(h->S.bus_of_ibus, st));
    CK(h->active.alloc(nS));
    CK(h->err.alloc(nS));
    CK(h->iters.alloc(nS));
    CK(h->status.alloc(nS));
    CK(h->n_active.alloc(1));
    CK(h->J.alloc(nS));
    CK(h->laststep.alloc(nS));
    CK(h->maxstep.alloc(nS));
    CK(h->stop.alloc(1));
    CK(h->clk.alloc(6));
    CK(h->clk_acc.alloc(4));
    CK(h->steps_dev.alloc(1));
    CK(cudaMallocHost((void **)&h->h_n_active, sizeof(int)));
    CK(cudaMallocHost((void **)&h->h_stop, sizeof(StopRule)));
    // measurement-function tables in canonical numbering
    {
        const int L = h->S.L;
        std::vector<int> fr(net->from_bus, net->from_bus + L), to(net->to_bus, net->to_bus + L);
        std::vector<double> g(L), b(L), bh(L);
        for (int l = 0; l < L; ++l) {
            const double den = net->r[l] * net->r[l] + net->x[l] * net->x[l];
            g[l] = net->r[l] / den;
            b[l] = -net->x[l] / den;
            bh[l] = 0.5 * net->b_charge[l];
        }
        std::vector<int> beg(N + 1, 0), br;
        for (int l = 0; l < L; ++l) {
            ++beg[fr[l] + 1];
            ++beg[to[l] + 1];
        }
        for (int i = 0; i < N; ++i) beg[i + 1] += beg[i];
        br.assign(beg[N], 0);
        std::vector<int> fill(beg.begin(), beg.end() - 1);
        for (int l = 0; l < L; ++l) {
            br[fill[fr[l]]++] = l;
            br[fill[to[l]]++] = l;
        }
        // measurement values at the flat start (Vm = 1, Va = 0), internal row
        // order: Vm rows 1, active power rows 0, a reactive flow is -b_c/2 at
        // its end and a reactive injection the sum over the incident branches
        {
            std::vector<double> hc((size_t)3 * N + 4 * (size_t)L, 0.0), hi(M);
            for (int i = 0; i < N; ++i) hc[i] = 1.0;
            for (int l = 0; l < L; ++l) {
                hc[2 * (size_t)N + fr[l]] -= bh[l];
                hc[2 * (size_t)N + to[l]] -= bh[l];
                hc[3 * (size_t)N + (size_t)L + l] = -bh[l];       // Qf
                hc[3 * (size_t)N + 3 * (size_t)L + l] = -bh[l];   // Qt
            }
            for (int r = 0; r < M; ++r) hi[r] = hc[h->S.zperm[r]];
            CK(h->h_flat.upload(hi, st));
        }
        CK(h->m_from.upload(fr, st));
        CK(h->m_to.upload(to, st));
        CK(h->m_g.upload(g, st));
        CK(h->m_b.upload(b, st));
        CK(h->m_bh.upload(bh, st));
        CK(h->m_inc_beg.upload(beg, st));
        CK(h->m_inc_br.upload(br, st));
    }
    rc = h->opt.precision == MASE_MIXED ? autotune<float, float>(h.get()) : autotune<double, double>(h.get());
    if (rc != MASE_OK) return rc;
    rc = upload_measurements(h.get(), meas);
    if (rc != MASE_OK) return rc;
    CK(cudaStreamSynchronize(st));
    rc = join_out(h.get());
    if (rc != MASE_OK) return rc;
    *out = h.release();
    return MASE_OK;
}

int mase_set_measurements(mase_handle *h, const mase_measurements *meas) {
    if (!h || !meas) return set_err(MASE_EINVAL, "null argument");
    if (meas->n_snap != h->n_snap) return set_err(MASE_EINVAL, "n_snap differs from the handle's");
    CK(cudaSetDevice(h->opt.device));
    int rc = join_in(h);
    if (rc != MASE_OK) return rc;
    rc = upload_measurements(h, meas);
    int rc2 = join_out(h);
    return rc != MASE_OK ? rc : rc2;
}

int mase_solve(mase_handle *h, const double *x0, double tol, int32_t max_iter, double *x_out,
               mase_stats *stats) {
    if (!h) return set_err(MASE_EINVAL, "null handle");
    if (!h->has_z) return set_err(MASE_ENOTREADY, "no measurements set");
    if (max_iter < 1 || max_iter > 1000) return set_err(MASE_EINVAL, "max_iter out of range");
    if (!(tol >= 0.0)) return set_err(MASE_EINVAL, "tol must be >= 0");
    CK(cudaSetDevice(h->opt.device));
    int rc = join_in(h);
    if (rc != MASE_OK) return rc;
    rc = h->opt.precision == MASE_MIXED ? solve_impl<float, float>(h, x0, tol, max_iter, x_out, stats)
                                        : solve_impl<double, double>(h, x0, tol, max_iter, x_out, stats);
    int rc2 = join_out(h);
    return rc != MASE_OK ? rc : rc2;
}

int mase_measure(mase_handle *h, const double *x, int32_t n_snap, double *z_out) {
    if (!h || !x || !z_out || n_snap < 1) return set_err(MASE_EINVAL, "bad argument");
    CK(cudaSetDevice(h->opt.device));
    {
        int rc0 = join_in(h);
        if (rc0 != MASE_OK) return rc0;
    }
    cudaStream_t st = h->stream;
    const int N = h->S.N, L = h->S.L, M = h->S.m;
    const bool dx = is_device_ptr(x), dz = is_device_ptr(z_out);
    DevBuf<double> xs, zs;
    const double *xd = x;
    double *zd = z_out;
    if (!dx) {
        CK(xs.alloc((size_t)2 * N * n_snap));
        CK(cudaMemcpyAsync(xs.p, x, (size_t)2 * N * n_snap * sizeof(double), cudaMemcpyHostToDevice, st));
        xd = xs.p;
    }
    if (!dz) {
        CK(zs.alloc((size_t)M * n_snap));
        zd = zs.p;
    }
    k_measure<<<2048, 256, 0, st>>>(xd, zd, N, L, n_snap, h->m_from.p, h->m_to.p, h->m_g.p,
                                    h->m_b.p, h->m_bh.p, h->m_inc_beg.p, h->m_inc_br.p);
    CK(cudaGetLastError());
    if (!dz)
        CK(cudaMemcpyAsync(z_out, zd, (size_t)M * n_snap * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return join_out(h);
}

int mase_get_info(const mase_handle *h, mase_info *info) {
    if (!h || !info) return set_err(MASE_EINVAL, "null argument");
    *info = h->info;
    return MASE_OK;
}

int mase_set_start_mode(mase_handle *h, int32_t mode) {
    if (!h) return set_err(MASE_EINVAL, "null handle");
    if (mode != MASE_START_FLAT && mode != MASE_START_X0 && mode != MASE_START_LEARNED)
        return set_err(MASE_EINVAL, "bad start mode");
    h->start_mode = mode;
    return MASE_OK;
}

void mase_destroy(mase_handle *h) { delete h; }

}  // extern "C"

namespace mase_internal {

void set_last_error(const std::string &msg) { g_last_error = msg; }

bool coord_view(const mase_handle *h, CoordView &v) {
    if (!h) return false;
    v.precision = h->opt.precision;
    v.refine = h->opt.precision == MASE_MIXED ? h->opt.refine : 0;
    v.n_snap = h->n_snap;
    v.n_area = h->S.K;
    v.threads = h->threads;
    v.device = h->opt.device;
    v.smem_bnd = h->smem_bnd;
    v.T = h->T;
    v.B = h->bnd;
    v.off_B.resize(h->S.K);
    v.n_bnd.resize(h->S.K);
    for (int k = 0; k < h->S.K; ++k) {
        v.off_B[k] = h->S.areas[k].F.off_B;
        v.n_bnd[k] = h->S.areas[k].n_bnd;
    }
    v.xg_of_b = h->S.B.xg_of_b;
    v.stream = h->stream;
    v.user_stream = h->user_stream;
    v.ev_in = h->ev_in;
    v.ev_out = h->ev_out;
    return true;
}

}  // namespace mase_internal

namespace mase_internal {

void launch_objective(mase_handle *h, double *xV, double *xT, double *J, int *launches) {
    State X = make_state(h);
    X.xV = xV;
    X.xT = xT;
    X.J = J;
    auto kern = h->vec_global ? k_objective<true> : k_objective<false>;
    kern<<<h->S.K * h->n_snap, 256, h->smem_obj, h->stream>>>(h->d_areas.p, h->T, X, h->d_inst.p,
                                                               h->vscratch.p);
    if (launches) ++*launches;
}

}  // namespace mase_internal
