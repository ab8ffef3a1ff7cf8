// Potts kernel buckets (flat DAG: one node per end-label), storage f16 (with the floor of the labelling at 2^-24).
#include "pfm_solver.cuh"

namespace pfm {

SolverBase* make_potts_f16(int maxl, int dim, const ProblemView& v) {
#define PFM_POTTS(L, DM) \
    if (maxl == L && dim == DM) return new Solver<L, L, DM, false, __half>(v);
    PFM_POTTS(4, 2) PFM_POTTS(4, 3) PFM_POTTS(8, 2) PFM_POTTS(8, 3) PFM_POTTS(16, 2) PFM_POTTS(16, 3)
#undef PFM_POTTS
    return nullptr;
}

BatchBase* make_batch_potts_f16(int maxl, int dim) {
#define PFM_BPOTTS(L, DM) \
    if (maxl == L && dim == DM) return new BatchRunner<L, L, DM, false, __half>();
    PFM_BPOTTS(4, 2) PFM_BPOTTS(4, 3) PFM_BPOTTS(8, 2) PFM_BPOTTS(8, 3) PFM_BPOTTS(16, 2) PFM_BPOTTS(16, 3)
#undef PFM_BPOTTS
    return nullptr;
}

}  // namespace pfm
