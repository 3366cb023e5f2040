// Coordinator solve that allocates no device memory (mase_coordinator_noalloc).
//
// Some callers cannot call cudaMalloc when they need the coordinator step:
// a host program whose device memory belongs to another allocator (a
// framework's caching pool, or a pool carved out once at start-up) that does
// not allow raw allocations next to it, and latency-bound loops that must not
// take the device-wide synchronisation cudaMalloc and cudaFree can imply.
// This entry point lets them run the coordinator step on condensed blocks
// they already hold: its scratch (boundary-factor storage, the assembled copy
// used by the refinement, small index tables and a status word per snapshot)
// lives in one file-scope static device array of kScratchBytes, which every
// GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mase.h"
#define MASE_SHARED_TEMPLATES_ONLY
#include "internal.h"
#include "kernels.cuh"

using namespace mase_dev;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_coord_scratch[kScratchBytes];

int fail(int code, const std::string &msg) {
    mase_internal::set_last_error(msg);
    return code;
}

// Per-device device address of g_coord_scratch, resolved once per device with
// that device current (host code must not use the symbol's host-side name).
struct Slot {
    void *ptr = nullptr;
};
std::mutex g_mu;
Slot g_slots[kMaxDevices];

struct Tabs {
    const long long *blk_base;   // per area: first element of its S blocks
    const long long *rhs_base;   // per area: first element of its rhs blocks
    const int *off_B;            // per area: Schur-block offset in the instance storage
    const int *n_bnd;            // per area: local boundary unknowns
    const int *xg_of_b;          // boundary-system unknown -> x_Gamma index
    int *status;                 // per snapshot: 1 = non-SPD pivot, 2 = non-finite, 4 = a bounded wait gave up
};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

template <class RG, class RS>
__global__ void __launch_bounds__(512) k_coordinator_noalloc(Tables T, BndDev B, Tabs tb,
                                                             const double *__restrict__ Sin,
                                                             const double *__restrict__ bin,
                                                             double *__restrict__ dxg, RG *st_all,
                                                             RG *A_all, int refine) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_err;
    const int s = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x, nG = B.n_gamma;
    double *bhat = (double *)smem;
    double *x = bhat + nG;
    double *r = x + nG;
    RS *y = (RS *)(r + nG);
    RG *st = st_all + (long long)s * B.stride;
    RG *Am = A_all + (long long)s * B.stride;
    if (tid == 0) s_err = 0;
    // assembly S_Gamma = sum_k E_k^T S_b^k E_k from the caller's packed blocks
    for (int P = tid; P < B.F.store_total; P += nt) {
        double v = 0.0;
        for (int i = B.asm_beg[P]; i < B.asm_beg[P + 1]; ++i) {
            const int k = B.asm_area[i];
            const int nb = tb.n_bnd[k];
            const long long np = (long long)nb * (nb + 1) / 2;
            v += Sin[tb.blk_base[k] + s * np + (B.asm_off[i] - tb.off_B[k])];
        }
        st[P] = RG(v);
        Am[P] = RG(v);
    }
    for (int gi = tid; gi < nG; gi += nt) {
        double v = 0.0;
        for (int i = B.rhs_beg[gi]; i < B.rhs_beg[gi + 1]; ++i) {
            const int k = B.rhs_area[i];
            v += bin[tb.rhs_base[k] + (long long)s * tb.n_bnd[k] + B.rhs_lv[i]];
        }
        bhat[gi] = v;
        y[gi] = RS(v);
    }
    __syncthreads();
    factor_numeric<RG, RS>(B.F, T, FlatStore<RG>{st}, y, (int *)(smem + B.smem_off_ctr), &s_err);
    back_solve<RG, RS>(B.F, T, FlatStore<RG>{st}, y);
    for (int gi = tid; gi < nG; gi += nt) x[gi] = double(y[gi]);
    __syncthreads();
    for (int it = 0; it < refine; ++it) {
        for (int gi = tid; gi < nG; gi += nt) r[gi] = bhat[gi];
        __syncthreads();
        // r = b_hat - S_Gamma x, FP64 accumulation over the stored lower triangle
        boundary_residual<RG>(B.F, T, Am, x, r, BlockTeam());
        __syncthreads();
        for (int gi = tid; gi < nG; gi += nt) y[gi] = RS(r[gi]);
        __syncthreads();
        solve_forward<RG, RS>(B.F, T, FlatStore<RG>{st}, y);
        back_solve<RG, RS>(B.F, T, FlatStore<RG>{st}, y);
        for (int gi = tid; gi < nG; gi += nt) x[gi] += double(y[gi]);
        __syncthreads();
    }
    bool bad = false;
    for (int gi = tid; gi < nG; gi += nt) {
        const double d = x[gi];
        dxg[(long long)s * nG + tb.xg_of_b[gi]] = d;
        if (!isfinite(d)) bad = true;
    }
    if (bad) atomicOr(tb.status + s, 2);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(tb.status + s, s_err);
}

bool is_device(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int mase_coordinator_noalloc(mase_handle *h, const double *S_blocks, int64_t n_S,
                             const double *b_blocks, int64_t n_b, double *dx_gamma, int64_t n_dx) {
    using mase_internal::CoordView;
    CoordView v;
    if (!mase_internal::coord_view(h, v)) return fail(MASE_EINVAL, "null handle");
    if (!S_blocks || !b_blocks || !dx_gamma) return fail(MASE_EINVAL, "null argument");
    {
        // the element counts the handle implies, checked before any device work
        long long need_S = 0, need_b = 0;
        for (int k = 0; k < v.n_area; ++k) {
            const long long nb = v.n_bnd[k];
            need_S += nb * (nb + 1) / 2;
            need_b += nb;
        }
        need_S *= v.n_snap;
        need_b *= v.n_snap;
        const long long need_dx = (long long)v.n_snap * v.B.n_gamma;
        if (n_S != need_S || n_b != need_b || n_dx != need_dx)
            return fail(MASE_EINVAL, "element counts (S_blocks " + std::to_string(n_S) + ", b_blocks " +
                                         std::to_string(n_b) + ", dx_gamma " + std::to_string(n_dx) +
                                         ") differ from the handle's (" + std::to_string(need_S) + ", " +
                                         std::to_string(need_b) + ", " + std::to_string(need_dx) + ")");
    }
    if (v.device < 0 || v.device >= kMaxDevices) return fail(MASE_EINVAL, "device ordinal out of range");
    if (cudaSetDevice(v.device) != cudaSuccess) return fail(MASE_EDEVICE, "cudaSetDevice failed");
    if (!is_device(S_blocks) || !is_device(b_blocks) || !is_device(dx_gamma))
        return fail(MASE_EINVAL, "S_blocks, b_blocks and dx_gamma must be device pointers");
    const int S = v.n_snap, K = v.n_area, nG = v.B.n_gamma;
    if (nG == 0) return MASE_OK;
    const size_t rg = v.precision == MASE_MIXED ? sizeof(float) : sizeof(double);
    // scratch layout
    size_t o = 0;
    const size_t o_blk = o;
    o = up256(o + K * sizeof(long long));
    const size_t o_rhs = o;
    o = up256(o + K * sizeof(long long));
    const size_t o_offB = o;
    o = up256(o + K * sizeof(int));
    const size_t o_nb = o;
    o = up256(o + K * sizeof(int));
    const size_t o_xg = o;
    o = up256(o + nG * sizeof(int));
    const size_t o_status = o;
    o = up256(o + S * sizeof(int));
    const size_t tab_bytes = o;
    const size_t o_st = o;
    o = up256(o + (size_t)S * v.B.stride * rg);
    const size_t o_A = o;
    o = up256(o + (size_t)S * v.B.stride * rg);
    if (o > kScratchBytes)
        return fail(MASE_EINVAL, "coordinator needs " + std::to_string(o) +
                                     " bytes of scratch; the static maximum is " +
                                     std::to_string(kScratchBytes));
    // one-time set-up per device: device address of the static scratch
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        Slot &sl = g_slots[v.device];
        if (!sl.ptr) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_coord_scratch);
            if (e != cudaSuccess)
                return fail(MASE_EDEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            sl.ptr = p;
        }
        base = (unsigned char *)sl.ptr;
    }
    {
        cudaError_t ea = v.precision == MASE_MIXED
            ? cudaFuncSetAttribute(k_coordinator_noalloc<float, float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem_bnd)
            : cudaFuncSetAttribute(k_coordinator_noalloc<double, double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem_bnd);
        if (ea != cudaSuccess)
            return fail(MASE_EDEVICE, std::string("coordinator attributes: ") + cudaGetErrorString(ea));
    }
    // small index tables (host -> scratch)
    std::vector<unsigned char> host(tab_bytes, 0);
    long long acc_s = 0, acc_b = 0;
    for (int k = 0; k < K; ++k) {
        const long long nb = v.n_bnd[k];
        ((long long *)(host.data() + o_blk))[k] = acc_s;
        ((long long *)(host.data() + o_rhs))[k] = acc_b;
        ((int *)(host.data() + o_offB))[k] = v.off_B[k];
        ((int *)(host.data() + o_nb))[k] = (int)nb;
        acc_s += (long long)S * nb * (nb + 1) / 2;
        acc_b += (long long)S * nb;
    }
    std::memcpy(host.data() + o_xg, v.xg_of_b.data(), nG * sizeof(int));
    cudaStream_t st = v.stream;
    cudaError_t e;
    if ((e = cudaEventRecord(v.ev_in, v.user_stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, v.ev_in, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base, host.data(), tab_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(MASE_EDEVICE, std::string("coordinator set-up: ") + cudaGetErrorString(e));
    Tabs tb;
    tb.blk_base = (const long long *)(base + o_blk);
    tb.rhs_base = (const long long *)(base + o_rhs);
    tb.off_B = (const int *)(base + o_offB);
    tb.n_bnd = (const int *)(base + o_nb);
    tb.xg_of_b = (const int *)(base + o_xg);
    tb.status = (int *)(base + o_status);
    if (v.precision == MASE_MIXED)
        k_coordinator_noalloc<float, float><<<S, v.threads, v.smem_bnd, st>>>(
            v.T, v.B, tb, S_blocks, b_blocks, dx_gamma, (float *)(base + o_st), (float *)(base + o_A),
            v.refine);
    else
        k_coordinator_noalloc<double, double><<<S, v.threads, v.smem_bnd, st>>>(
            v.T, v.B, tb, S_blocks, b_blocks, dx_gamma, (double *)(base + o_st),
            (double *)(base + o_A), v.refine);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(MASE_EDEVICE, std::string("coordinator launch: ") + cudaGetErrorString(e));
    std::vector<int> status(S, 0);
    if ((e = cudaMemcpyAsync(status.data(), base + o_status, S * sizeof(int), cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess ||
        (e = cudaEventRecord(v.ev_out, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(v.user_stream, v.ev_out, 0)) != cudaSuccess)
        return fail(MASE_EDEVICE, std::string("coordinator: ") + cudaGetErrorString(e));
    // the worst status over all snapshots, whatever their order
    int any = 0;
    for (int s = 0; s < S; ++s) any |= status[s];
    if (any & 4) return fail(MASE_EDEVICE, "a bounded device-side wait gave up");
    if (any & 1) return fail(MASE_EUNOBSERVABLE, "non-positive pivot in the boundary system");
    if (any & 2) return fail(MASE_ENONFINITE, "non-finite boundary step");
    return MASE_OK;
}

}  // extern "C"
