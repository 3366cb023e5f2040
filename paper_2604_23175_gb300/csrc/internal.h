// Read-only view of a handle's coordinator data for entry points that live
// in other translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.cuh"

struct mase_handle;

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
