// Definitions shared by the library's translation units: the handle, device
// buffers, and views of the handle for entry points in other files.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/mase.h"
#include "kernels.cuh"

#include "setup.h"

namespace mase_internal {

struct HostTables {
    std::vector<int> sn_c0, sn_w, sn_nr, sn_off, sn_order, lev_off;
    std::vector<int> rows, rel;
    std::vector<int> locbus, qvarV, qvarT, own_q, own_gvv, own_ebeg;
    std::vector<int> end_qi, end_qj, end_own, end_var, end_gpos;
    std::vector<double> end_g, end_b, end_bh;
    std::vector<int> item_pos, ebnd;
    std::vector<int> tasks, lev_tasks, item_rec, chunk_rec, lev_chunks;
};

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count) {
        release();
        n = count;
        if (!count) return cudaSuccess;
        return cudaMalloc((void **)&p, count * sizeof(T));
    }
    cudaError_t upload(const std::vector<T> &v, cudaStream_t st) {
        cudaError_t e = alloc(v.size());
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    }
};

// true for device or managed memory (asks the CUDA runtime)
bool is_device_pointer(const void *p);

struct WarmStart;                       // per-area MLP warm start (warmstart.cu)
void destroy_warmstart(WarmStart *w);
// Fills (xV, xT) with the learned start for the handle's current measurements
// and keeps, per snapshot, whichever of the learned and the flat start has
// the lower objective.  Returns a MASE_* code.
int learned_start(mase_handle *h, int *launches);
// per snapshot, 1 where the last learned start kept the networks' proposal
const int *learned_picked(const mase_handle *h);
// device flag set when a tensor-core GEMM of the learned start gave up a
// bounded wait (nullptr before the first learned start)
int *learned_gemm_err(const mase_handle *h);
// Adds r^T W r at the states (xV, xT) to J[s] for every snapshot (area kernel
// in objective mode); J must be zeroed by the caller.
void launch_objective(mase_handle *h, double *xV, double *xT, double *J, int *launches);

}  // namespace mase_internal

using mase_internal::DevBuf;
using mase_internal::HostTables;
using mase_dev::AreaDev;
using mase_dev::BndDev;
using mase_dev::StopRule;
using mase_dev::Tables;

// One launch of the area kernel over a class of (area, snapshot) instances
// that share a block size and a dynamic shared-memory size.
struct LocalClass {
    int threads = 512;
    size_t smem = 0;
    int n_areas = 0;
    std::vector<int2> inst_h;
    DevBuf<int2> inst;
};

struct mase_handle {
    mase::Setup S;
    mase_options opt{};
    cudaStream_t stream = nullptr;
    int n_snap = 0;
    int start_mode = MASE_START_FLAT;
    int smem_limit = 0;
    int threads = 256;
    // tables
    HostTables H;
    std::vector<AreaDev> areas_h;
    BndDev bnd{};
    DevBuf<AreaDev> d_areas;
    DevBuf<int> t_sn_c0, t_sn_w, t_sn_nr, t_sn_off, t_sn_order,
        t_lev_off, t_rows, t_rel, t_locbus, t_qvarV, t_qvarT, t_own_q,
        t_own_gvv, t_own_ebeg, t_end_qi, t_end_qj, t_end_own, t_end_var, t_end_gpos,
        t_item_pos, t_ebnd,
        t_tasks, t_lev_tasks, t_item_rec, t_chunk_rec, t_lev_chunks;
    DevBuf<double> t_end_g, t_end_b, t_end_bh;
    DevBuf<int> b_asm_beg, b_asm_area, b_asm_off, b_rhs_beg, b_rhs_area, b_rhs_lv, b_bvar_ibus,
        b_bvar_isT, b_asm_str, b_rhs_str;
    DevBuf<long long> b_asm_abs, b_rhs_abs;
    Tables T{};
    DevBuf<int2> d_inst;
    std::vector<int2> inst_h;
    // state and measurements
    DevBuf<double> xV, xT, z_int, z_stage, W;
    DevBuf<uint8_t> mask_int, mask_stage;
    bool has_mask = false, has_z = false;
    DevBuf<int> zperm, bus_of_ibus;
    DevBuf<double> h_flat;   // h(x) at the flat start, internal row order
    // work buffers
    DevBuf<unsigned char> fac, cvec, bst, bA;
    DevBuf<double> bh, dxG, J, laststep, xbuf;
    DevBuf<double> dx_zero;   // a zero boundary step for the inner local iterations
    DevBuf<int> active, err, iters, status, n_active;
    DevBuf<unsigned long long> maxstep;
    int *h_n_active = nullptr;   // pinned
    DevBuf<int> restart;         // [S] snapshots of a flat-start fallback
    size_t smem_local = 0, smem_back = 0, smem_bnd = 0, smem_obj = 0;
    // launch configuration (autotuned at create when options.autotune)
    std::vector<std::unique_ptr<LocalClass>> lcls;   // area-kernel launch classes
    std::vector<int> area_order;                     // areas by descending estimated work
    int back_threads = 256;
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // concurrent class launches
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    // areas whose vectors live in global scratch (one area holding a large network)
    int vec_global = 0;
    long long vscratch_bytes = 0;
    DevBuf<unsigned char> vscratch;
    // coordinator on 2-block clusters (the whole boundary factor on chip)
    int bnd_cluster = 0;
    size_t smem_bnd_cl = 0;
    long long fac_elems = 0, c_elems = 0, bh_elems = 0;
    // measurement function tables (canonical numbering)
    DevBuf<int> m_from, m_to, m_inc_beg, m_inc_br;
    DevBuf<double> m_g, m_b, m_bh;
    // graph
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;
    int graph_launches = 0;
    DevBuf<StopRule> stop;
    cudaStream_t user_stream = nullptr;   // caller's stream (NULL = legacy default stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_solve[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_stage[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // options.profile
    // device-side loop control and stage clocks
    cudaGraphConditionalHandle loop_cond = 0;
    DevBuf<unsigned long long> clk;
    DevBuf<double> clk_acc;
    DevBuf<int> steps_dev;
    StopRule *h_stop = nullptr;   // pinned
    mase_info info{};
    mase_internal::WarmStart *ws = nullptr;   // learned warm start, if trained or loaded
    DevBuf<double> xV2, xT2;                  // learned start kept while the flat start's J is formed

    ~mase_handle() {
        mase_internal::destroy_warmstart(ws);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (h_n_active) cudaFreeHost(h_n_active);
        if (h_stop) cudaFreeHost(h_stop);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        for (auto &e : ev_solve)
            if (e) cudaEventDestroy(e);
        for (auto &e : ev_stage)
            if (e) cudaEventDestroy(e);
        if (stream) cudaStreamDestroy(stream);
        for (auto &q : side)
            if (q) cudaStreamDestroy(q);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (auto &e : ev_join)
            if (e) cudaEventDestroy(e);
    }
};

namespace mase_internal {

struct CoordView {
    int precision;                    // MASE_FP64 | MASE_MIXED
    int refine;
    int n_snap, n_area, threads, device;
    size_t smem_bnd;
    mase_dev::Tables T;
    mase_dev::BndDev B;
    std::vector<int> off_B, n_bnd;    // per area: Schur block offset, local boundary size
    std::vector<int> xg_of_b;         // boundary-system unknown -> x_Gamma index
    cudaStream_t stream, user_stream;
    cudaEvent_t ev_in, ev_out;
};

bool coord_view(const mase_handle *h, CoordView &v);

// Sets the message returned by mase_last_error() on this thread.
void set_last_error(const std::string &msg);

}  // namespace mase_internal
