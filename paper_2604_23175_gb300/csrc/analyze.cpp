// Host-only entry points: structural analysis and self-check of the one-time
// symbolic setup (Sec. 4.1, 4.3).  No CUDA call is made here, so both work on
// a machine without a GPU.
#include <algorithm>
#include <cstring>
#include <string>

#include "../../include/mase.h"
#include "setup.h"

namespace {
thread_local std::string g_analyze_error;

int build_from(const mase_network *net, const mase_partition *part, mase::Setup &S) {
    if (!net || !part) {
        g_analyze_error = "null argument";
        return MASE_EINVAL;
    }
    mase::NetIn ni{net->n_bus, net->n_branch, net->slack_bus, net->from_bus, net->to_bus,
                   net->r, net->x, net->b_charge};
    if (!mase::build_setup(ni, part->n_area, part->area_of_bus, S)) {
        g_analyze_error = S.error;
        return MASE_EINVAL;
    }
    return MASE_OK;
}
}  // namespace

extern "C" {

int mase_analyze(const mase_network *net, const mase_partition *part, mase_info *info) {
    if (!info) return MASE_EINVAL;
    mase::Setup S;
    int rc = build_from(net, part, S);
    if (rc != MASE_OK) return rc;
    std::memset(info, 0, sizeof(*info));
    info->n_bus = S.N;
    info->n_branch = S.L;
    info->n_area = S.K;
    info->n_meas = S.m;
    info->n_state = 2 * S.N - 1;
    info->n_boundary_bus = S.n_boundary_bus;
    info->n_gamma = S.B.n_gamma;
    for (const auto &A : S.areas) {
        info->max_area_vars = std::max(info->max_area_vars, A.n_int + A.n_bnd);
        info->max_area_nb = std::max(info->max_area_nb, A.n_bnd);
        info->factor_nnz += A.F.store_total;
        info->local_flops += A.F.flops;
        info->g_updates += A.g_updates;
        info->n_supernodes += A.F.nsn();
        info->n_units += (int64_t)A.F.unit_sn.size();
        info->max_levels = std::max(info->max_levels, A.F.nlev());
        info->max_area_store = std::max(info->max_area_store, A.F.store_total);
        info->coord_S_elems += (int64_t)A.n_bnd * (A.n_bnd + 1) / 2;
        info->coord_b_elems += A.n_bnd;
    }
    info->boundary_store = S.B.F.store_total;
    info->boundary_levels = S.B.F.nlev();
    info->boundary_flops = S.B.F.flops;
    return MASE_OK;
}

int mase_selfcheck(const mase_network *net, const mase_partition *part, uint64_t seed,
                   double *errors4) {
    if (!errors4) return MASE_EINVAL;
    mase::Setup S;
    int rc = build_from(net, part, S);
    if (rc != MASE_OK) return rc;
    std::string err;
    if (!mase::selfcheck(S, seed, errors4, err)) {
        g_analyze_error = err;
        return MASE_EINVAL;
    }
    return MASE_OK;
}

const char *mase_analyze_error(void) { return g_analyze_error.c_str(); }

void mase_abi_sizes(int64_t *sizes4) {
    if (!sizes4) return;
    sizes4[0] = (int64_t)sizeof(mase_options);
    sizes4[1] = (int64_t)sizeof(mase_stats);
    sizes4[2] = (int64_t)sizeof(mase_info);
    sizes4[3] = (int64_t)sizeof(mase_warmstart_options);
}

}  // extern "C"
