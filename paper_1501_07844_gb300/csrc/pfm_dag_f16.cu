// DAG / HMF kernel buckets (path-weight form of Algorithm 2), storage f16 (with the floor of the labelling at 2^-24).
#include "pfm_solver.cuh"

namespace pfm {

SolverBase* make_dag_f16(int maxl, int maxn, int dim, const ProblemView& v) {
#define PFM_DAG(L, N, DM) \
    if (maxl == L && maxn == N && dim == DM) return new Solver<L, N, DM, true, __half>(v);
    PFM_DAG(8, 12, 2) PFM_DAG(8, 12, 3) PFM_DAG(16, 16, 2) PFM_DAG(16, 16, 3)
#undef PFM_DAG
    return nullptr;
}

BatchBase* make_batch_dag_f16(int maxl, int maxn, int dim) {
#define PFM_BDAG(L, N, DM) \
    if (maxl == L && maxn == N && dim == DM) return new BatchRunner<L, N, DM, true, __half>();
    PFM_BDAG(8, 12, 2) PFM_BDAG(8, 12, 3) PFM_BDAG(16, 16, 2) PFM_BDAG(16, 16, 3)
#undef PFM_BDAG
    return nullptr;
}

BatchBase* make_batch_dag_tma_f16(const BatchMember* m, int n, int dim) {
    if (dim == 3) return BatchDagTma<3, __half>::fits(m, n) ? new BatchDagTma<3, __half>() : nullptr;
    if (dim == 2) return BatchDagTma<2, __half>::fits(m, n) ? new BatchDagTma<2, __half>() : nullptr;
    return nullptr;
}

BatchBase* make_batch_dag4_tma_f16(const BatchMember* m, int n, int dim) {
    if (dim == 3) return BatchDag4Tma<3, __half>::fits(m, n) ? new BatchDag4Tma<3, __half>() : nullptr;
    if (dim == 2) return BatchDag4Tma<2, __half>::fits(m, n) ? new BatchDag4Tma<2, __half>() : nullptr;
    return nullptr;
}

}  // namespace pfm
