/*
 * pfm_oracle.c -- plain FP64 CPU oracle for the pseudo-flow continuous
 * max-flow method (Baxter, Rajchl, Yuan, Peters, arXiv 1501.07844).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the solver.  Every function
 * performs the paper's steps in the paper's order as whole-grid sweeps, with
 * no blocking or fusion, so that each line can be checked against the paper
 * by eye.  The conventions are listed in pfm_oracle.h.
 *
 * Parity-unpinned part: the LIMIT POINT of the ORC_PAPER_LITERAL variant
 * (flow step on the unnormalised labelling), where that iteration stalls
 * short of the optimum.  Its iterations themselves are pinned by
 * hand-worked two-voxel examples of Algorithms 1, 2 and 3, its invariants
 * (simplex, capacity) and its S = 0 closed form.
 */
#include "pfm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

long orc_nvox(const orc_grid* g) { return g->nx * g->ny * g->nz; }

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double cap(const double* S_field, const double* s_node, int node, long i) {
    double s = s_node ? s_node[node] : 1.0;
    if (S_field) s *= S_field[i];
    return s;
}

/* ---------------------------------------------------------------------------
 * Discrete operators.  The paper takes the flow step "in the manner of
 * Chambolle" (Eq. potts_flowupdate) without fixing a discretisation; the
 * standard forward-difference gradient and its negative adjoint are used.
 * ------------------------------------------------------------------------- */

/* Forward-difference gradient, zero at the last index of each axis. */
void orc_grad(const orc_grid* g, const double* u, double* out) {
    const long nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
#pragma omp parallel for schedule(static) if (nz * ny * nx > 65536)
    for (long zy = 0; zy < nz * ny; ++zy) {
        const long z = zy / ny, y = zy % ny;
        for (long x = 0; x < nx; ++x) {
            const long i = zy * nx + x;
            out[i] = (x < nx - 1) ? u[i + 1] - u[i] : 0.0;
            out[n + i] = (y < ny - 1) ? u[i + nx] - u[i] : 0.0;
            if (g->ndim == 3) out[2 * n + i] = (z < nz - 1) ? u[i + nx * ny] - u[i] : 0.0;
        }
    }
}

/* Divergence = -(gradient)^T: backward difference of each component, the
 * component counted as zero at index -1 and at the last index of its axis. */
void orc_div(const orc_grid* g, const double* q, double* out) {
    const long nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
#pragma omp parallel for schedule(static) if (nz * ny * nx > 65536)
    for (long zy = 0; zy < nz * ny; ++zy) {
        const long z = zy / ny, y = zy % ny;
        for (long x = 0; x < nx; ++x) {
            const long i = zy * nx + x;
            double s = 0.0;
            s += (x < nx - 1 ? q[i] : 0.0) - (x > 0 ? q[i - 1] : 0.0);
            s += (y < ny - 1 ? q[n + i] : 0.0) - (y > 0 ? q[n + i - nx] : 0.0);
            if (g->ndim == 3)
                s += (z < nz - 1 ? q[2 * n + i] : 0.0) - (z > 0 ? q[2 * n + i - nx * ny] : 0.0);
            out[i] = s;
        }
    }
}

/* Projection onto the capacity set {|q| <= s} (the Proj of
 * Eq. potts_flowupdate and of the primal constraint |q_L(x)| <= S_L(x)). */
void orc_project(int ndim, int norm, double s, double* y) {
    if (norm == ORC_ISO) {
        double r2 = 0.0;
        for (int k = 0; k < ndim; ++k) r2 += y[k] * y[k];
        const double r = sqrt(r2);
        if (r > s) {
            const double f = s / r;
            for (int k = 0; k < ndim; ++k) y[k] *= f;
        }
    } else {
        for (int k = 0; k < ndim; ++k) {
            if (y[k] > s) y[k] = s;
            if (y[k] < -s) y[k] = -s;
        }
    }
}

/* One projected gradient step q <- Proj(q - step * grad f) for one node's
 * flow field (Eq. potts_flowupdate; Algorithm 1 flow line; Algorithm 2
 * bottom-up flow line). */
static void flow_step(const orc_grid* g, int norm, double step, const double* f,
                      const double* S_field, const double* s_node, int node,
                      double* qn /* [ndim][n] */, double* gbuf /* [ndim][n] */) {
    const long n = orc_nvox(g);
    const int nd = g->ndim;
    orc_grad(g, f, gbuf);
#pragma omp parallel for schedule(static) if (n > 65536)
    for (long i = 0; i < n; ++i) {
        double y[3];
        for (int k = 0; k < nd; ++k) y[k] = qn[k * n + i] - step * gbuf[k * n + i];
        orc_project(nd, norm, cap(S_field, s_node, node, i), y);
        for (int k = 0; k < nd; ++k) qn[k * n + i] = y[k];
    }
}

static double vnorm(int nd, int norm, const double* gk, long n, long i) {
    double s = 0.0;
    if (norm == ORC_ISO) {
        for (int k = 0; k < nd; ++k) s += gk[k * n + i] * gk[k * n + i];
        return sqrt(s);
    }
    for (int k = 0; k < nd; ++k) s += fabs(gk[k * n + i]);
    return s;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1: pseudo-flow continuous Potts model.
 * ------------------------------------------------------------------------- */

/* Initialisation: u_L = 1/#L (Algorithm 1, first line); the paper does not
 * initialise q, it is read as zero. */
void orc_potts_init(const orc_grid* g, int nl, double* u, double* q) {
    const long n = orc_nvox(g);
    for (long i = 0; i < (long)nl * n; ++i) u[i] = 1.0 / nl;
    memset(q, 0, sizeof(double) * (size_t)nl * g->ndim * n);
}

static void potts_normalise(long n, int nl, double* u) {
    /* a(x) = sum_L u_L(x); u_L(x) <- u_L(x) / a(x)  (Algorithm 1, last two lines) */
#pragma omp parallel for schedule(static) if (n > 65536)
    for (long i = 0; i < n; ++i) {
        double a = 0.0;
        for (int L = 0; L < nl; ++L) a += u[(long)L * n + i];
        for (int L = 0; L < nl; ++L) u[(long)L * n + i] /= a;
    }
}

void orc_potts_iterate(const orc_grid* g, int nl, const double* D,
                       const double* S_field, const double* s_node,
                       const orc_params* p, int iters, double* u, double* q) {
    const long n = orc_nvox(g);
    const int nd = g->ndim;
    double* dv = (double*)malloc(sizeof(double) * n);
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    for (int it = 0; it < iters; ++it) {
        /* u_L <- u_L exp(-(D_L + div q_L)/c)   (Algorithm 1, first loop line) */
        for (int L = 0; L < nl; ++L) {
            orc_div(g, q + (long)L * nd * n, dv);
            double* uL = u + (long)L * n;
            const double* DL = D + (long)L * n;
#pragma omp parallel for schedule(static) if (n > 65536)
            for (long i = 0; i < n; ++i) uL[i] *= exp(-(DL[i] + dv[i]) / p->c);
        }
        if (p->grad_source == ORC_PAPER_LITERAL) {
            /* q_L <- Proj(q_L - c tau grad u_L) on the unnormalised u, then normalise. */
            for (int L = 0; L < nl; ++L)
                flow_step(g, p->norm, p->c * p->tau, u + (long)L * n, S_field, s_node, L,
                          q + (long)L * nd * n, gb);
            potts_normalise(n, nl, u);
        } else {
            /* Normalise first, then the flow step on the normalised u (the
             * gradient of Eq. potts_bregmanopt with respect to div q_L). */
            potts_normalise(n, nl, u);
            for (int L = 0; L < nl; ++L)
                flow_step(g, p->norm, p->c * p->tau, u + (long)L * n, S_field, s_node, L,
                          q + (long)L * nd * n, gb);
        }
    }
    free(dv);
    free(gb);
}

/* E(u) of Eq. potts_original with per-label capacity S_L(x) (the
 * "variable smoothness" form of the primal max-flow Eq. potts_primal) and
 * the pseudo-flow dual P(q) = sum_x min_L (D_L + div q_L) of Eq. potts_pseudo. */
void orc_potts_energy(const orc_grid* g, int nl, const double* D,
                      const double* S_field, const double* s_node, int norm,
                      const double* u, const double* q,
                      double* primal, double* dual) {
    const long n = orc_nvox(g);
    const int nd = g->ndim;
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    double* z = (double*)malloc(sizeof(double) * (size_t)nl * n);
    double E = 0.0;
    for (int L = 0; L < nl; ++L) {
        const double* uL = u + (long)L * n;
        const double* DL = D + (long)L * n;
        orc_grad(g, uL, gb);
        double e = 0.0;
#pragma omp parallel for reduction(+ : e) schedule(static) if (n > 65536)
        for (long i = 0; i < n; ++i)
            e += DL[i] * uL[i] + cap(S_field, s_node, L, i) * vnorm(nd, norm, gb, n, i);
        E += e;
        orc_div(g, q + (long)L * nd * n, z + (long)L * n);
#pragma omp parallel for schedule(static) if (n > 65536)
        for (long i = 0; i < n; ++i) z[(long)L * n + i] += DL[i];
    }
    double P = 0.0;
#pragma omp parallel for reduction(+ : P) schedule(static) if (n > 65536)
    for (long i = 0; i < n; ++i) {
        double m = z[i];
        for (int L = 1; L < nl; ++L) m = fmin(m, z[(long)L * n + i]);
        P += m;
    }
    *primal = E;
    *dual = P;
    free(gb);
    free(z);
}

/* ---------------------------------------------------------------------------
 * Algorithm 2: pseudo-flow DAGMF (HMF is the tree special case).
 * ------------------------------------------------------------------------- */

typedef struct {
    int nn, nleaf;
    int* order;     /* top-down topological order of the non-source nodes */
    int* leaf_of;   /* node -> leaf index or -1 */
    int* is_leaf;
} dag_info;

static void dag_free(dag_info* di) {
    free(di->order);
    free(di->leaf_of);
    free(di->is_leaf);
}

/* Validates the DAG and builds the order O (Kahn's algorithm from S). */
static int dag_build(const orc_dag* dag, dag_info* di) {
    const int nn = dag->n_nodes, ne = dag->n_edges;
    di->nn = nn;
    di->order = (int*)calloc(nn > 0 ? nn : 1, sizeof(int));
    di->leaf_of = (int*)calloc(nn > 0 ? nn : 1, sizeof(int));
    di->is_leaf = (int*)calloc(nn > 0 ? nn : 1, sizeof(int));
    int* indeg = (int*)calloc(nn > 0 ? nn : 1, sizeof(int));
    int* nchild = (int*)calloc(nn > 0 ? nn : 1, sizeof(int));
    int ok = nn > 0;
    for (int e = 0; e < ne && ok; ++e) {
        const int a = dag->parent[e], b = dag->child[e];
        if (a < -1 || a >= nn || b < 0 || b >= nn || a == b) ok = 0;
        else {
            indeg[b]++;
            if (a >= 0) nchild[a]++;
        }
    }
    int cnt = 0;
    if (ok) {
        /* every node must have at least one parent (S or a node) */
        for (int v = 0; v < nn; ++v)
            if (indeg[v] == 0) ok = 0;
    }
    if (ok) {
        /* Kahn: edges from S are satisfied at the start */
        int* rem = (int*)calloc(nn, sizeof(int));
        for (int e = 0; e < ne; ++e)
            if (dag->parent[e] >= 0) rem[dag->child[e]]++;
        int head = 0;
        for (int v = 0; v < nn; ++v)
            if (rem[v] == 0) di->order[cnt++] = v;
        while (head < cnt) {
            const int v = di->order[head++];
            for (int e = 0; e < ne; ++e)
                if (dag->parent[e] == v && --rem[dag->child[e]] == 0)
                    di->order[cnt++] = dag->child[e];
        }
        free(rem);
        if (cnt != nn) ok = 0; /* cycle */
    }
    di->nleaf = 0;
    if (ok) {
        for (int v = 0; v < nn; ++v) {
            di->is_leaf[v] = nchild[v] == 0;
            di->leaf_of[v] = di->is_leaf[v] ? di->nleaf++ : -1;
        }
        if (di->nleaf == 0) ok = 0;
    }
    free(indeg);
    free(nchild);
    if (!ok) {
        dag_free(di);
        return -1;
    }
    return 0;
}

int orc_dag_n_leaves(const orc_dag* dag) {
    dag_info di;
    if (dag_build(dag, &di)) return -1;
    const int r = di.nleaf;
    dag_free(&di);
    return r;
}

/* Path weights W_(A,B) = sum over paths A -> B of the product of edge
 * weights, by the recursion of Section 3.3 (W_(A,A) = 1, W_(A,B) =
 * sum_{L in A.C} w_(A,L) W_(L,B)).  Row A, column B. */
int orc_dag_path_weights(const orc_dag* dag, double* W) {
    dag_info di;
    if (dag_build(dag, &di)) return -1;
    const int nn = di.nn;
    memset(W, 0, sizeof(double) * nn * nn);
    /* process A bottom-up so that every child's row is complete */
    for (int k = nn - 1; k >= 0; --k) {
        const int A = di.order[k];
        W[A * nn + A] = 1.0;
        for (int e = 0; e < dag->n_edges; ++e)
            if (dag->parent[e] == A)
                for (int B = 0; B < nn; ++B)
                    W[A * nn + B] += dag->w[e] * W[dag->child[e] * nn + B];
    }
    dag_free(&di);
    return 0;
}

/* u_L = 1/|L| on end-labels (Algorithm 2, first line); q = 0. */
int orc_dag_init(const orc_grid* g, const orc_dag* dag, double* u, double* q) {
    dag_info di;
    if (dag_build(dag, &di)) return -1;
    const long n = orc_nvox(g);
    for (long i = 0; i < (long)di.nleaf * n; ++i) u[i] = 1.0 / di.nleaf;
    memset(q, 0, sizeof(double) * (size_t)di.nn * g->ndim * n);
    dag_free(&di);
    return 0;
}

/* Top-down flow excess (definition of d_L in Section 3.3; Algorithm 2,
 * first three lines of the loop): d_A = div q_A (+ D_A on end-labels), then
 * in order O every node passes w * d to its children. */
static void dag_excess(const orc_grid* g, const orc_dag* dag, const dag_info* di,
                       const double* D, const double* q, double* d) {
    const long n = orc_nvox(g);
    const int nd = g->ndim;
    for (int A = 0; A < di->nn; ++A) orc_div(g, q + (long)A * nd * n, d + (long)A * n);
    for (int A = 0; A < di->nn; ++A)
        if (di->is_leaf[A]) {
            const double* DL = D + (long)di->leaf_of[A] * n;
#pragma omp parallel for schedule(static) if (n > 65536)
            for (long i = 0; i < n; ++i) d[(long)A * n + i] += DL[i];
        }
    for (int k = 0; k < di->nn; ++k) {
        const int A = di->order[k];
        for (int e = 0; e < dag->n_edges; ++e)
            if (dag->parent[e] == A) {
                double* dc = d + (long)dag->child[e] * n;
                const double* da = d + (long)A * n;
                const double w = dag->w[e];
#pragma omp parallel for schedule(static) if (n > 65536)
                for (long i = 0; i < n; ++i) dc[i] += w * da[i];
            }
    }
}

int orc_dag_iterate(const orc_grid* g, const orc_dag* dag, const double* D,
                    const double* S_field, const double* s_node,
                    const orc_params* p, int iters, double* u, double* q) {
    dag_info di;
    if (dag_build(dag, &di)) return -1;
    const long n = orc_nvox(g);
    const int nd = g->ndim, nn = di.nn, nl = di.nleaf;
    double* d = (double*)malloc(sizeof(double) * (size_t)nn * n);
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    for (int it = 0; it < iters; ++it) {
        dag_excess(g, dag, &di, D, q, d);
        /* end-labels: u_L <- u_L exp(-d_L / c) */
        for (int A = 0; A < nn; ++A)
            if (di.is_leaf[A]) {
                double* uL = u + (long)di.leaf_of[A] * n;
                const double* dA = d + (long)A * n;
#pragma omp parallel for schedule(static) if (n > 65536)
                for (long i = 0; i < n; ++i) uL[i] *= exp(-dA[i] / p->c);
            }
        if (p->grad_source == ORC_PAPER_LITERAL) {
            /* d_L <- u_L before normalising, as printed */
            for (int A = 0; A < nn; ++A)
                if (di.is_leaf[A]) memcpy(d + (long)A * n, u + (long)di.leaf_of[A] * n, sizeof(double) * n);
            potts_normalise(n, nl, u);
        } else {
            potts_normalise(n, nl, u);
            for (int A = 0; A < nn; ++A)
                if (di.is_leaf[A]) memcpy(d + (long)A * n, u + (long)di.leaf_of[A] * n, sizeof(double) * n);
        }
        /* non-end-labels: d_L <- 0 */
        for (int A = 0; A < nn; ++A)
            if (!di.is_leaf[A]) memset(d + (long)A * n, 0, sizeof(double) * n);
        /* order O^-1: flow step of A, then pass w * d_A up to A's parents */
        for (int k = nn - 1; k >= 0; --k) {
            const int A = di.order[k];
            flow_step(g, p->norm, p->c * p->tau, d + (long)A * n, S_field, s_node, A,
                      q + (long)A * nd * n, gb);
            for (int e = 0; e < dag->n_edges; ++e)
                if (dag->child[e] == A && dag->parent[e] >= 0) {
                    double* dp = d + (long)dag->parent[e] * n;
                    const double* da = d + (long)A * n;
                    const double w = dag->w[e];
#pragma omp parallel for schedule(static) if (n > 65536)
                    for (long i = 0; i < n; ++i) dp[i] += w * da[i];
                }
        }
    }
    free(d);
    free(gb);
    dag_free(&di);
    return 0;
}

/* E(u) of Eq. dagmf_original: every non-source node carries its smoothness
 * term, inner labellings follow u_A = sum_{L in A.C} w_(A,L) u_L, data terms
 * sit on end-labels only.  Dual: P(q) = sum_x min_{L end-label} d_L(x)
 * (Eq. dagmf_pseudo). */
int orc_dag_energy(const orc_grid* g, const orc_dag* dag, const double* D,
                   const double* S_field, const double* s_node, int norm,
                   const double* u, const double* q,
                   double* primal, double* dual) {
    dag_info di;
    if (dag_build(dag, &di)) return -1;
    const long n = orc_nvox(g);
    const int nd = g->ndim, nn = di.nn;
    double* uA = (double*)calloc((size_t)nn * n, sizeof(double));
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    double* d = (double*)malloc(sizeof(double) * (size_t)nn * n);
    for (int A = 0; A < nn; ++A)
        if (di.is_leaf[A]) memcpy(uA + (long)A * n, u + (long)di.leaf_of[A] * n, sizeof(double) * n);
    for (int k = nn - 1; k >= 0; --k) {
        const int A = di.order[k];
        for (int e = 0; e < dag->n_edges; ++e)
            if (dag->child[e] == A && dag->parent[e] >= 0) {
                double* up = uA + (long)dag->parent[e] * n;
                const double* ua = uA + (long)A * n;
                const double w = dag->w[e];
#pragma omp parallel for schedule(static) if (n > 65536)
                for (long i = 0; i < n; ++i) up[i] += w * ua[i];
            }
    }
    double E = 0.0;
    for (int A = 0; A < nn; ++A) {
        orc_grad(g, uA + (long)A * n, gb);
        const double* DL = di.is_leaf[A] ? D + (long)di.leaf_of[A] * n : NULL;
        const double* ua = uA + (long)A * n;
        double e = 0.0;
#pragma omp parallel for reduction(+ : e) schedule(static) if (n > 65536)
        for (long i = 0; i < n; ++i)
            e += (DL ? DL[i] * ua[i] : 0.0) + cap(S_field, s_node, A, i) * vnorm(nd, norm, gb, n, i);
        E += e;
    }
    dag_excess(g, dag, &di, D, q, d);
    double P = 0.0;
#pragma omp parallel for reduction(+ : P) schedule(static) if (n > 65536)
    for (long i = 0; i < n; ++i) {
        double m = INFINITY;
        for (int A = 0; A < nn; ++A)
            if (di.is_leaf[A]) m = fmin(m, d[(long)A * n + i]);
        P += m;
    }
    *primal = E;
    *dual = P;
    free(uA);
    free(gb);
    free(d);
    dag_free(&di);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Algorithm 3: pseudo-flow continuous Ishikawa model.  nlev = N levels,
 * N+1 labels.  The excess of label L_i accumulates the divergences of the
 * flows of levels 1..i (top-down), the labelling is normalised over all
 * N+1 labels, and the flow of level i is driven by the sum of the labels
 * L_i..L_N (bottom-up accumulation).
 * ------------------------------------------------------------------------- */
void orc_ishikawa_init(const orc_grid* g, int nlev, double* u, double* q) {
    const long n = orc_nvox(g);
    for (long i = 0; i < (long)(nlev + 1) * n; ++i) u[i] = 1.0 / (nlev + 1);
    memset(q, 0, sizeof(double) * (size_t)nlev * g->ndim * n);
}

void orc_ishikawa_iterate(const orc_grid* g, int nlev, const double* D,
                          const double* S_field, const double* s_level,
                          const orc_params* p, int iters, double* u, double* q) {
    const long n = orc_nvox(g);
    const int nd = g->ndim, nlab = nlev + 1;
    double* d = (double*)malloc(sizeof(double) * (size_t)nlab * n);
    double* dv = (double*)malloc(sizeof(double) * n);
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    for (int it = 0; it < iters; ++it) {
        /* d_{L_0} = 0; d_{L_i} = d_{L_{i-1}} + div q_{L_i} for i = 1..N */
#pragma omp parallel for schedule(static) if (n > 65536)
        for (long x = 0; x < n; ++x) d[x] = 0.0;
        for (int i = 1; i <= nlev; ++i) {
            orc_div(g, q + (long)(i - 1) * nd * n, dv);
#pragma omp parallel for schedule(static) if (n > 65536)
            for (long x = 0; x < n; ++x) d[(long)i * n + x] = d[(long)(i - 1) * n + x] + dv[x];
        }
        /* d_{L_i} += D_{L_i} for every label */
#pragma omp parallel for schedule(static) if (n > 65536)
        for (long k = 0; k < (long)nlab * n; ++k) d[k] += D[k];
        /* u_{L_i} <- u_{L_i} exp(-d_{L_i}/c) */
#pragma omp parallel for schedule(static) if (n > 65536)
        for (long k = 0; k < (long)nlab * n; ++k) u[k] *= exp(-d[k] / p->c);
        if (p->grad_source == ORC_PAPER_LITERAL) {
            memcpy(d, u, sizeof(double) * (size_t)nlab * n); /* d <- u before normalising */
            potts_normalise(n, nlab, u);
        } else {
            potts_normalise(n, nlab, u);
            memcpy(d, u, sizeof(double) * (size_t)nlab * n);
        }
        /* d_{L_i} += d_{L_{i+1}} for i = N-1 .. 1 */
        for (int i = nlev - 1; i >= 1; --i) {
#pragma omp parallel for schedule(static) if (n > 65536)
            for (long x = 0; x < n; ++x) d[(long)i * n + x] += d[(long)(i + 1) * n + x];
        }
        /* q_{L_i} <- Proj(q_{L_i} - c tau grad d_{L_i}) for i = 1..N */
        for (int i = 1; i <= nlev; ++i)
            flow_step(g, p->norm, p->c * p->tau, d + (long)i * n, S_field, s_level, i - 1,
                      q + (long)(i - 1) * nd * n, gb);
    }
    free(d);
    free(dv);
    free(gb);
}

/* ---------------------------------------------------------------------------
 * Explicit-flow augmented Lagrangian continuous max-flow (Potts).
 *
 * Primal Eq. potts_primal: maximise sum_x p_S s.t. p_L <= D_L, |q_L| <= S_L,
 * G_L := div q_L - p_S + p_L = 0, with multipliers u_L (Eq. potts_primaldual).
 * Augmented Lagrangian  sum p_S + sum_L <u_L, G_L> - (gamma/2) sum_L |G_L|^2,
 * maximised block by block, then u_L <- u_L - gamma G_L:
 *   q_L : one projected ascent step; the gradient of the augmented terms
 *         with respect to q_L is -grad(u_L - gamma G_L);
 *   p_L : p_L = min(D_L, p_S - div q_L + u_L/gamma)  (closed form);
 *   p_S : p_S = (sum_L (div q_L + p_L - u_L/gamma) + 1/gamma) / #L.
 * ------------------------------------------------------------------------- */
void orc_alm_potts_init(const orc_grid* g, int nl, const double* D,
                        double* u, double* q, double* pS, double* pL) {
    const long n = orc_nvox(g);
    for (long i = 0; i < n; ++i) {
        double m = D[i];
        for (int L = 1; L < nl; ++L) m = fmin(m, D[(long)L * n + i]);
        pS[i] = m;
        for (int L = 0; L < nl; ++L) {
            pL[(long)L * n + i] = m;
            u[(long)L * n + i] = 1.0 / nl;
        }
    }
    memset(q, 0, sizeof(double) * (size_t)nl * g->ndim * n);
}

void orc_alm_potts_iterate(const orc_grid* g, int nl, const double* D,
                           const double* S_field, const double* s_node,
                           int norm, double gamma, double step, int iters,
                           double* u, double* q, double* pS, double* pL,
                           double* flow_value) {
    const long n = orc_nvox(g);
    const int nd = g->ndim;
    double* dv = (double*)malloc(sizeof(double) * (size_t)nl * n);
    double* f = (double*)malloc(sizeof(double) * n);
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    for (int it = 0; it < iters; ++it) {
        for (int L = 0; L < nl; ++L) {
            double* qL = q + (long)L * nd * n;
            double* dL = dv + (long)L * n;
            double* pl = pL + (long)L * n;
            const double* uL = u + (long)L * n;
            const double* DL = D + (long)L * n;
            orc_div(g, qL, dL);
            for (long i = 0; i < n; ++i) f[i] = uL[i] - gamma * (dL[i] - pS[i] + pl[i]);
            /* ascent along +(-grad f): q <- Proj(q - step * grad f) */
            flow_step(g, norm, step, f, S_field, s_node, L, qL, gb);
            orc_div(g, qL, dL);
            for (long i = 0; i < n; ++i) pl[i] = fmin(DL[i], pS[i] - dL[i] + uL[i] / gamma);
        }
        for (long i = 0; i < n; ++i) {
            double s = 0.0;
            for (int L = 0; L < nl; ++L)
                s += dv[(long)L * n + i] + pL[(long)L * n + i] - u[(long)L * n + i] / gamma;
            pS[i] = (s + 1.0 / gamma) / nl;
        }
        for (int L = 0; L < nl; ++L)
            for (long i = 0; i < n; ++i)
                u[(long)L * n + i] -= gamma * (dv[(long)L * n + i] - pS[i] + pL[(long)L * n + i]);
    }
    double fv = 0.0;
    for (long i = 0; i < n; ++i) fv += pS[i];
    *flow_value = fv;
    free(dv);
    free(f);
    free(gb);
}

/* ---------------------------------------------------------------------------
 * Exhaustive search over binary labellings of the two-label Potts energy
 * E(u) = sum_x D_0 u_0 + D_1 u_1 + sum_L S_L |grad u_L|, u_1 = 1 - u_0.
 * ------------------------------------------------------------------------- */
int orc_bruteforce_binary(const orc_grid* g, const double* D,
                          const double* S_field, const double* s_node, int norm,
                          double* best, double* second, unsigned char* label0) {
    const long n = orc_nvox(g);
    if (n > 24) return -1;
    const int nd = g->ndim;
    double* u = (double*)malloc(sizeof(double) * 2 * n);
    double* gb = (double*)malloc(sizeof(double) * nd * n);
    double b1 = INFINITY, b2 = INFINITY;
    unsigned long arg = 0;
    for (unsigned long m = 0; m < (1ul << n); ++m) {
        for (long i = 0; i < n; ++i) {
            u[i] = (double)((m >> i) & 1ul);
            u[n + i] = 1.0 - u[i];
        }
        double E = 0.0;
        for (int L = 0; L < 2; ++L) {
            orc_grad(g, u + (long)L * n, gb);
            for (long i = 0; i < n; ++i)
                E += D[(long)L * n + i] * u[(long)L * n + i] + cap(S_field, s_node, L, i) * vnorm(nd, norm, gb, n, i);
        }
        if (E < b1) {
            b2 = b1;
            b1 = E;
            arg = m;
        } else if (E < b2) {
            b2 = E;
        }
    }
    for (long i = 0; i < n; ++i) label0[i] = (unsigned char)((arg >> i) & 1ul);
    *best = b1;
    *second = b2;
    free(u);
    free(gb);
    return 0;
}
