/*
 * pfm_oracle.h -- plain FP64 CPU oracle for the pseudo-flow continuous
 * max-flow method of Baxter, Rajchl, Yuan and Peters (arXiv 1501.07844).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  The CUDA solver shares
 * no code, header, table or helper with it.
 *
 * Conventions (the paper leaves the discretisation open; these readings are
 * stated once here and followed by every function):
 *   - grid of nx*ny*nz voxels, unit spacing, x fastest: index (z*ny+y)*nx+x;
 *     a 2-D problem has nz == 1 and ndim == 2 (flows have ndim components);
 *   - gradient: forward difference, zero at the last index of each axis;
 *   - divergence: the negative adjoint of that gradient (backward
 *     difference, flow component treated as zero at index -1 and at the
 *     last index of its axis);
 *   - capacity set: Euclidean ball |q| <= S (ORC_ISO) or the box
 *     |q_i| <= S (ORC_ANISO, whose dual norm is the l1 norm);
 *   - arrays are label-major: u[leaf][voxel], D[leaf][voxel],
 *     q[node][component][voxel];
 *   - capacity of node A at voxel x: s_node[A] * S_field[x], either factor
 *     may be NULL (then 1).
 */
#ifndef PFM_ORACLE_H
#define PFM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ISO = 0, ORC_ANISO = 1 };
/* Which labelling the flow step differentiates: the normalised u (the
 * gradient of the smoothed objective, Eq. potts_bregmanopt) or the
 * unnormalised u*exp(-(D+div q)/c) exactly as Algorithm 1 prints it. */
enum { ORC_NORMALISED = 0, ORC_PAPER_LITERAL = 1 };

typedef struct {
    int ndim;          /* 2 or 3 */
    long nx, ny, nz;   /* nz == 1 when ndim == 2 */
} orc_grid;

typedef struct {
    double c;          /* entropic weight c > 0 */
    double tau;        /* gradient step tau > 0 (applied step is c*tau) */
    int norm;          /* ORC_ISO or ORC_ANISO */
    int grad_source;   /* ORC_NORMALISED or ORC_PAPER_LITERAL */
} orc_params;

/* Label DAG (Section 3.3): non-source nodes 0..n_nodes-1, edges
 * parent -> child with weight w; parent == -1 is the source S. */
typedef struct {
    int n_nodes;
    int n_edges;
    const int* parent;
    const int* child;
    const double* w;
} orc_dag;

long orc_nvox(const orc_grid* g);
/* Number of OpenMP threads the sweeps use (1 without OpenMP). */
int orc_threads(void);

/* Discrete operators. */
void orc_grad(const orc_grid* g, const double* u, double* out /* [ndim][n] */);
void orc_div(const orc_grid* g, const double* q /* [ndim][n] */, double* out);
void orc_project(int ndim, int norm, double s, double* y /* [ndim] */);

/* Algorithm 1 (continuous Potts).  u: [nl][n] in/out, q: [nl][ndim][n] in/out.
 * Initialise with orc_potts_init (u = 1/nl, q = 0). */
void orc_potts_init(const orc_grid* g, int nl, double* u, double* q);
void orc_potts_iterate(const orc_grid* g, int nl, const double* D,
                       const double* S_field, const double* s_node,
                       const orc_params* p, int iters, double* u, double* q);
/* Primal energy (Eq. potts_original) and pseudo-flow dual (Eq. potts_pseudo). */
void orc_potts_energy(const orc_grid* g, int nl, const double* D,
                      const double* S_field, const double* s_node, int norm,
                      const double* u, const double* q,
                      double* primal, double* dual);

/* Algorithm 2 (DAGMF; HMF is the tree case).  Returns 0 on success,
 * -1 for a malformed DAG (cycle, bad index, no leaf).  Leaves are the nodes
 * without children, ordered by ascending node id; u: [n_leaf][n],
 * D: [n_leaf][n], q: [n_nodes][ndim][n]. */
int orc_dag_n_leaves(const orc_dag* dag);
int orc_dag_path_weights(const orc_dag* dag, double* W /* [n_nodes][n_nodes] */);
int orc_dag_init(const orc_grid* g, const orc_dag* dag, double* u, double* q);
int orc_dag_iterate(const orc_grid* g, const orc_dag* dag, const double* D,
                    const double* S_field, const double* s_node,
                    const orc_params* p, int iters, double* u, double* q);
int orc_dag_energy(const orc_grid* g, const orc_dag* dag, const double* D,
                   const double* S_field, const double* s_node, int norm,
                   const double* u, const double* q,
                   double* primal, double* dual);

/* Algorithm 3 (continuous Ishikawa model): N+1 ordered labels L_0..L_N,
 * N flow fields q_{L_1}..q_{L_N} with per-level capacities s_level[i-1]
 * (times S_field), u: [N+1][n], q: [N][ndim][n], D: [N+1][n]. */
void orc_ishikawa_init(const orc_grid* g, int nlev, double* u, double* q);
void orc_ishikawa_iterate(const orc_grid* g, int nlev, const double* D,
                          const double* S_field, const double* s_level,
                          const orc_params* p, int iters, double* u, double* q);

/* Explicit-flow ("full-flow") augmented-Lagrangian continuous max-flow for
 * the Potts model (primal Eq. potts_primal, multipliers u of
 * Eq. potts_primaldual).  Independent algorithm used to pin the optimum.
 * State: u[nl][n], q[nl][ndim][n], pS[n], pL[nl][n].  On return *flow_value
 * holds the integral of p_S. */
void orc_alm_potts_init(const orc_grid* g, int nl, const double* D,
                        double* u, double* q, double* pS, double* pL);
void orc_alm_potts_iterate(const orc_grid* g, int nl, const double* D,
                           const double* S_field, const double* s_node,
                           int norm, double gamma, double step, int iters,
                           double* u, double* q, double* pS, double* pL,
                           double* flow_value);

/* Exhaustive minimum of the two-label Potts energy over binary labellings
 * (n <= 24 voxels).  Writes the minimum, the second-best energy of any
 * different labelling, and the minimising labelling (1 = label 0). */
int orc_bruteforce_binary(const orc_grid* g, const double* D /* [2][n] */,
                          const double* S_field, const double* s_node, int norm,
                          double* best, double* second, unsigned char* label0);

#ifdef __cplusplus
}
#endif
#endif
