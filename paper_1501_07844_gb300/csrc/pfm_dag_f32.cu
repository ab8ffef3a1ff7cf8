// DAG / HMF kernel buckets (path-weight form of Algorithm 2), storage f32.
#include "pfm_solver.cuh"

namespace pfm {

SolverBase* make_dag_f32(int maxl, int maxn, int dim, const ProblemView& v) {
#define PFM_DAG(L, N, DM) \
    if (maxl == L && maxn == N && dim == DM) return new Solver<L, N, DM, true, float>(v);
    PFM_DAG(8, 12, 2) PFM_DAG(8, 12, 3) PFM_DAG(16, 16, 2) PFM_DAG(16, 16, 3)
#undef PFM_DAG
    return nullptr;
}

BatchBase* make_batch_dag_f32(int maxl, int maxn, int dim) {
#define PFM_BDAG(L, N, DM) \
    if (maxl == L && maxn == N && dim == DM) return new BatchRunner<L, N, DM, true, float>();
    PFM_BDAG(8, 12, 2) PFM_BDAG(8, 12, 3) PFM_BDAG(16, 16, 2) PFM_BDAG(16, 16, 3)
#undef PFM_BDAG
    return nullptr;
}

BatchBase* make_batch_dag_tma_f32(const BatchMember* m, int n, int dim) {
    if (dim == 3) return BatchDagTma<3, float>::fits(m, n) ? new BatchDagTma<3, float>() : nullptr;
    if (dim == 2) return BatchDagTma<2, float>::fits(m, n) ? new BatchDagTma<2, float>() : nullptr;
    return nullptr;
}

BatchBase* make_batch_dag4_tma_f32(const BatchMember* m, int n, int dim) {
    if (dim == 3) return BatchDag4Tma<3, float>::fits(m, n) ? new BatchDag4Tma<3, float>() : nullptr;
    if (dim == 2) return BatchDag4Tma<2, float>::fits(m, n) ? new BatchDag4Tma<2, float>() : nullptr;
    return nullptr;
}

}  // namespace pfm
