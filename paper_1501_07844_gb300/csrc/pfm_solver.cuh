// pfm_solver.cuh -- host-side launch logic per kernel bucket.
//
// A bucket fixes at compile time the register-array sizes (MAXL end-labels,
// MAXN nodes), the spatial dimension and the storage type; the actual
// counts are runtime values <= the bucket maxima.
#pragma once

#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "pfm_device.cuh"
#include "pfm_tma.cuh"
#include "pfm_tma_dag.cuh"
#include "pfm_tma_inplace.cuh"
#include "pfm_tma_ishikawa.cuh"
#include "pfm_tma_dag4.cuh"
#include "pfm_tma_energy4.cuh"
#include "pfm_tma_tree.cuh"
#include "pfm_tma_x2.cuh"

namespace pfm {

// Encodes a tiled TMA descriptor (pfm_api.cu; driver entry point looked up
// through the runtime).  dims / box are innermost first; strides in bytes
// for dims 1..rank-1.  Returns false if the CUDA driver rejects the map.
bool encode_tiled_map(CUtensorMap* map, const void* base, int elem_bytes, int rank, const unsigned long long* dims,
                      const unsigned long long* strides, const unsigned* box);

// What a solver bucket needs from the problem (filled by the C-ABI layer).
struct ProblemView {
    int ndim, nx, ny, nz, nl, nn;
    int px;        // row pitch (elements) of every state / data array
    long long n;   // slots per label / component: px*ny*nz
    float c, tau;
    int literal, aniso;
    const float* D;
    const float* S;
    float* abuf;
    unsigned* flags;
    const float* s_node;   // host [nn]
    const float* W;        // host [nn][nl] path weights (DAG) or nullptr
};

// Host side of the TMA DAG kernels.  Sparse path-weight lists over the
// flow-carrying nodes (nodes from nf on have zero capacity and identically
// zero flow) and the shared-memory layout; false if three stages do not fit
// in the 227 KB a CTA may use (dynamic + the lists staged statically).
inline bool build_dag_lists(const StepArgs<DMAX, DMAX>& a, int dim, int es, DagLists* lists, DagTmaLayout* lay) {
    if ((a.px * es) % 16 != 0 || (a.px * 4) % 16 != 0) return false;
    int nf = 1;
    for (int A = 0; A < a.nn; ++A)
        if (a.s_node[A] > 0.f) nf = A + 1;
    *lay = DagTmaLayout(a.nl, nf, dim, es);
    if (lay->total + (int)sizeof(DagLists) + 64 > 227 * 1024) return false;
    *lists = DagLists{};
    lists->nf = nf;
    for (int A = 0; A < nf; ++A)
        for (int j = 0; j < a.nl; ++j)
            if (a.W[A][j] != 0.f) {
                lists->anc[j][lists->anc_n[j]] = (unsigned char)A;
                lists->anc_w[j][lists->anc_n[j]++] = a.W[A][j];
                lists->desc[A][lists->desc_n[A]] = (unsigned char)j;
                lists->desc_w[A][lists->desc_n[A]++] = a.W[A][j];
            }
    return true;
}

// Two-level label trees (source -> inner nodes -> end-labels), recognised
// from the path weights W_(A,j) (node A, end-label j): an inner node's row
// has two or more nonzeros (its end-labels); the own node of end-label j has
// W = 1 at j only; an end-label under an inner node with no other child
// shares its one-entry row with that node (the two are interchangeable:
// same excess, same driving field); one under the source alone has no
// parent node.  Groups: the inner nodes with their end-labels (at most
// four each), single-child chains, and the source's own end-labels packed
// four to a group; at most four groups.  False for anything else (deeper
// trees, end-labels with two parents) and when three stages of every
// node's flows do not fit in shared memory.
inline bool build_tree_shape(const StepArgs<DMAX, DMAX>& a, int dim, int es, TreeShape* ts) {
    const int nl = a.nl, nn = a.nn;
    if (nl < 1 || nn > DMAX || nl > DMAX) return false;
    const TreeTmaLayout lay(nl, nn, dim, es);
    if (lay.total + 64 > 227 * 1024) return false;
    int cnt[DMAX] = {0};
    for (int A = 0; A < nn; ++A)
        for (int j = 0; j < nl; ++j) cnt[A] += a.W[A][j] != 0.f;
    int cover[DMAX];  // inner node (>= 2 end-labels) above end-label j, or -1
    for (int j = 0; j < nl; ++j) cover[j] = -1;
    bool used[DMAX] = {false};
    *ts = TreeShape{};
    int ng = 0;
    auto add_group = [&](int inner) {
        if (ng >= TREE_MAXG) return -1;
        ts->inner[ng] = inner;
        ts->n[ng] = 0;
        return ng++;
    };
    // inner nodes with two or more end-labels: disjoint supports
    for (int A = 0; A < nn; ++A) {
        if (cnt[A] < 2) continue;
        if (cnt[A] > TREE_FAN) return false;
        const int g = add_group(A);
        if (g < 0) return false;
        used[A] = true;
        for (int j = 0; j < nl; ++j)
            if (a.W[A][j] != 0.f) {
                if (cover[j] >= 0) return false;  // two parents, or nested inner nodes
                cover[j] = A;
            }
    }
    // the own node of every end-label (and single-child chains)
    int lnode_of[DMAX], chain_of[DMAX];
    for (int j = 0; j < nl; ++j) {
        lnode_of[j] = chain_of[j] = -1;
        for (int A = 0; A < nn; ++A) {
            if (cnt[A] != 1 || a.W[A][j] == 0.f) continue;
            if (lnode_of[j] < 0 && a.W[A][j] == 1.0f)
                lnode_of[j] = A;
            else if (chain_of[j] < 0)
                chain_of[j] = A;
            else
                return false;  // a chain of three or more nodes above j
        }
        if (lnode_of[j] < 0) return false;
        if (chain_of[j] >= 0 && cover[j] >= 0) return false;
        used[lnode_of[j]] = true;
        if (chain_of[j] >= 0) used[chain_of[j]] = true;
    }
    for (int A = 0; A < nn; ++A)
        if (!used[A]) return false;
    auto add_leaf = [&](int g, int j, float w) {
        const int h = ts->n[g]++;
        ts->leaf[g][h] = j;
        ts->lnode[g][h] = lnode_of[j];
        ts->w[g][h] = w;
    };
    for (int g = 0; g < ng; ++g)
        for (int j = 0; j < nl; ++j)
            if (cover[j] == ts->inner[g]) add_leaf(g, j, a.W[ts->inner[g]][j]);
    int direct = -1;  // group of end-labels under the source (no parent flow)
    for (int j = 0; j < nl; ++j) {
        if (cover[j] >= 0) continue;
        if (chain_of[j] >= 0) {
            const int g = add_group(chain_of[j]);
            if (g < 0) return false;
            add_leaf(g, j, a.W[chain_of[j]][j]);
        } else {
            if (direct < 0 || ts->n[direct] == TREE_FAN) direct = add_group(-1);
            if (direct < 0) return false;
            add_leaf(direct, j, 0.f);
        }
    }
    ts->ng = ng;
    return true;
}

// DAGs with at most four non-end-label nodes, recognised from the path
// weights W_(A,j): every end-label j has its own node (a row with W = 1 at j
// and zero elsewhere; of a single-child chain, whose two rows are equal, one
// node is taken as the end-label's and the other as an inner node -- they
// enter the excess and the accumulation alike); every other node is an inner
// node, at most four, and at most twelve end-labels.  False otherwise, and
// when three stages of every node's flows do not fit in shared memory.
inline bool build_dag4_shape(const StepArgs<DMAX, DMAX>& a, int dim, int es, Dag4Shape* sh) {
    const int nl = a.nl, nn = a.nn;
    if (nl < 1 || nl > DAG4_MAXL || nn > DMAX) return false;
    const TreeTmaLayout lay(nl, nn, dim, es);
    if (lay.total + 64 > 227 * 1024) return false;
    *sh = Dag4Shape{};
    bool own[DMAX] = {false};
    for (int j = 0; j < nl; ++j) {
        int pick = -1;
        for (int A = nn - 1; A >= 0 && pick < 0; --A) {
            if (own[A] || a.W[A][j] != 1.0f) continue;
            bool single = true;
            for (int i = 0; i < nl && single; ++i) single = i == j || a.W[A][i] == 0.f;
            if (single) pick = A;
        }
        if (pick < 0) return false;
        own[pick] = true;
        sh->lnode[j] = pick;
    }
    sh->ni = 0;
    for (int k = 0; k < DAG4_INNER; ++k) sh->inner[k] = -1;
    for (int A = 0; A < nn; ++A) {
        if (own[A]) continue;
        if (sh->ni == DAG4_INNER) return false;
        const int k = sh->ni++;
        sh->inner[k] = A;
        for (int j = 0; j < nl; ++j) sh->w[j][k] = a.W[A][j];
    }
    return true;
}

// Tensor maps of one parity of a DAG problem: logical extents, pitched
// strides; the flow box covers the nf flow-carrying nodes.
// The flow-carrying nodes 0..nf-1 are the N = nl - 1 levels of an Ishikawa
// model (node k-1 is level k): every path weight W_(node k-1, L_j) is 1 for
// j >= k and 0 below (Algorithm 3's cumulative excess and accumulation),
// with at most 8 labels.
template <int MAXL, int MAXN>
inline bool is_ishikawa_chain(const StepArgs<MAXL, MAXN>& a) {
    int nf = 0;
    for (int A = 0; A < a.nn; ++A)
        if (a.s_node[A] > 0.f) nf = A + 1;
    if (a.nl < 2 || a.nl > ISH_MAXL || nf != a.nl - 1) return false;
    for (int A = 0; A < nf; ++A)
        for (int j = 0; j < a.nl; ++j)
            if (a.W[A][j] != (j > A ? 1.0f : 0.0f)) return false;
    return true;
}

// Maps of the Ishikawa kernel: the Potts kernel's boxes (32 x 8 tiles) over
// the nl labels and the flows of the nl - 1 levels (nodes 0..nl-2).
template <int MAXL, int MAXN>
inline bool encode_ishikawa_maps(const StepArgs<MAXL, MAXN>& a, int es, const void* u, const void* q,
                                 const float* D, const float* S, TmaMaps* m) {
    constexpr int DIM = 3;
    const int qbx = FTX + 2 * (16 / es);
    const unsigned long long nx = a.nx, ny = a.ny, nz = a.nz, px = a.px;
    const unsigned long long dims_u[4] = {nx, ny, nz, (unsigned long long)a.nl};
    const unsigned long long dims_q[4] = {nx, ny, nz, (unsigned long long)DIM * a.nn};
    const unsigned long long st_t[3] = {px * es, px * ny * es, px * ny * nz * es};
    const unsigned long long st_f[3] = {px * 4, px * ny * 4, px * ny * nz * 4};
    const unsigned box_u[4] = {(unsigned)TMA_BX, (unsigned)TMA_UY, 1u, (unsigned)a.nl};
    const unsigned box_q[4] = {(unsigned)qbx, (unsigned)TMA_QY, 1u, (unsigned)(DIM * (a.nl - 1))};
    const unsigned long long dims_s[3] = {nx, ny, nz};
    const unsigned box_s[3] = {(unsigned)FTX, (unsigned)FTY, 1u};
    if (!encode_tiled_map(&m->u, u, es, 4, dims_u, st_t, box_u)) return false;
    if (!encode_tiled_map(&m->q, q, es, 4, dims_q, st_t, box_q)) return false;
    if (!encode_tiled_map(&m->D, D, 4, 4, dims_u, st_f, box_u)) return false;
    if (S) return encode_tiled_map(&m->S, S, 4, 3, dims_s, st_f, box_s);
    m->S = m->D;  // never read: the kernel skips S when the problem has no field
    return true;
}

inline bool encode_dag_maps(const StepArgs<DMAX, DMAX>& a, int dim, int es, int nf, const void* u, const void* q,
                            const float* D, const float* S, TmaMaps* m, int qbx = 0) {
    if (qbx == 0) qbx = FTX + 2 * (16 / es);
    const unsigned long long nx = a.nx, ny = a.ny, nz = a.nz, px = a.px;
    const unsigned long long dims_u[4] = {nx, ny, nz, (unsigned long long)a.nl};
    const unsigned long long dims_q[4] = {nx, ny, nz, (unsigned long long)dim * a.nn};
    const unsigned long long st_t[3] = {px * es, px * ny * es, px * ny * nz * es};
    const unsigned long long st_f[3] = {px * 4, px * ny * 4, px * ny * nz * 4};
    const unsigned box_u[4] = {(unsigned)TMA_BX, (unsigned)DAG_UY, 1u, (unsigned)a.nl};
    const unsigned box_q[4] = {(unsigned)qbx, (unsigned)DAG_QY, 1u, (unsigned)(dim * nf)};
    const unsigned long long dims_s[3] = {nx, ny, nz};
    const unsigned box_s[3] = {(unsigned)FTX, (unsigned)DTY, 1u};
    if (!encode_tiled_map(&m->u, u, es, 4, dims_u, st_t, box_u)) return false;
    if (!encode_tiled_map(&m->q, q, es, 4, dims_q, st_t, box_q)) return false;
    if (!encode_tiled_map(&m->D, D, 4, 4, dims_u, st_f, box_u)) return false;
    if (S) return encode_tiled_map(&m->S, S, 4, 3, dims_s, st_f, box_s);
    m->S = m->D;  // never read: the kernel skips S when the problem has no field
    return true;
}

// Kernel arguments of a problem (one parity's buffers filled in by the caller).
template <int MAXL, int MAXN, bool IS_DAG>
StepArgs<MAXL, MAXN> make_step_args(const ProblemView& v, int zc) {
    StepArgs<MAXL, MAXN> a{};
    a.D = v.D;
    a.S = v.S;
    a.abuf = v.abuf;
    a.flags = v.flags;
    a.nx = v.nx;
    a.px = v.px;
    a.ny = v.ny;
    a.nz = v.nz;
    a.nl = v.nl;
    a.nn = v.nn;
    a.n = v.n;
    a.literal = v.literal;
    a.aniso = v.aniso;
    a.inv_c = 1.0f / v.c;
    a.ctau = v.c * v.tau;
    a.zc = zc;
    for (int A = 0; A < MAXN; ++A) a.s_node[A] = A < v.nn ? v.s_node[A] : 0.f;
    for (int A = 0; A < MAXN; ++A)
        for (int j = 0; j < MAXL; ++j) a.W[A][j] = (IS_DAG && A < v.nn && j < v.nl) ? v.W[A * v.nl + j] : 0.f;
    return a;
}

// The TMA DAG kernels (general, tree) take the arguments of the largest
// bucket; a problem of a smaller bucket is widened (entries past its counts
// are zero).
template <int MAXL, int MAXN>
StepArgs<DMAX, DMAX> widen_args(const StepArgs<MAXL, MAXN>& a) {
    static_assert(MAXL <= DMAX && MAXN <= DMAX, "bucket wider than the TMA DAG kernels");
    StepArgs<DMAX, DMAX> w{};
    w.u_in = a.u_in;
    w.u_out = a.u_out;
    w.q_in = a.q_in;
    w.q_out = a.q_out;
    w.D = a.D;
    w.S = a.S;
    w.abuf = a.abuf;
    w.flags = a.flags;
    w.nx = a.nx;
    w.ny = a.ny;
    w.nz = a.nz;
    w.nl = a.nl;
    w.nn = a.nn;
    w.px = a.px;
    w.literal = a.literal;
    w.aniso = a.aniso;
    w.zc = a.zc;
    w.n = a.n;
    w.inv_c = a.inv_c;
    w.ctau = a.ctau;
    for (int A = 0; A < MAXN; ++A) {
        w.s_node[A] = a.s_node[A];
        for (int j = 0; j < MAXL; ++j) w.W[A][j] = a.W[A][j];
    }
    return w;
}

struct SolverBase {
    virtual ~SolverBase() {}
    // One iteration reading (u_in, q_in) and writing (u_out, q_out); for the
    // in-place schedule u_in == u_out and q_in == q_out.  Returns the number
    // of kernels launched through *launches.
    // With partial != nullptr, a kernel that can also evaluates the energy
    // and dual of its input state into partial[2*k] and sets *nblocks = k;
    // *nblocks = 0 means it did not (the caller reduces separately).
    virtual cudaError_t step(const void* u_in, void* u_out, const void* q_in, void* q_out, bool fused,
                             int zc, cudaStream_t s, int* launches, double* partial = nullptr,
                             int* nblocks = nullptr) = 0;
    // Per-block (E, P) partials of the energy of (u, q) into partial[2*k];
    // *nblocks receives k (<= max_blocks).
    virtual cudaError_t energy(const void* u, const void* q, double* partial, int max_blocks, int zc, cudaStream_t s,
                               int* nblocks) = 0;
    // Number of partials the TMA energy kernel writes for chunk length zc (0 if it is not used).
    virtual long long tma_energy_blocks(int zc) const { return 0; }
    // Builds TMA descriptors for the double-buffered state; true if the
    // TMA-pipelined fused kernel can run on this problem.
    virtual bool prepare_tma(void* const* u, void* const* q, const float* D, const float* S) { return false; }
    // New data buffers (D, S) for later launches; the caller then prepares
    // the tensor maps over them again (prepare_tma).
    virtual void set_data(const float* D, const float* S) = 0;
    bool use_tma = true;  // cleared to force the register-staged fused kernel
    bool use_tree = true;  // cleared to run a two-level tree on the general TMA DAG kernel
    bool use_ishi = true;  // cleared to run an Ishikawa chain on the general TMA DAG kernel
    bool use_dag4 = true;  // cleared to run a DAG with <= 4 inner nodes on the general TMA DAG kernel
    // Forces the kernel family of the fused schedule ("fused_tma",
    // "fused_tma_ishikawa", "fused_tma_tree", "fused_tma_dag4",
    // "fused_tma_dag" or "fused", the register-staged kernel); false if the
    // problem cannot run it.
    virtual bool select(const char* name) = 0;
    bool use_tma_inplace = false;  // PFM_SCHEDULE_INPLACE: TMA-staged sweeps where available
    // Name of the kernel family step() launches for the given schedule.
    virtual const char* variant(bool fused) const = 0;
    // True if step() with a partials buffer evaluates the energy of its input.
    virtual bool fuses_energy(bool fused) const { return false; }
    // New entropic weight c and step tau for the following iterations.
    virtual void set_step(float c, float tau) = 0;
};

template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
struct Solver final : SolverBase {
    StepArgs<MAXL, MAXN> base{};
    size_t fused_smem = 0;
    static constexpr bool kTmaCapable = !IS_DAG && MAXL <= 8;
    static constexpr bool kDagTmaCapable = IS_DAG;  // every DAG bucket (arguments widened)
    bool tma_ready = false;
    const void* tma_u[2] = {nullptr, nullptr};
    TmaMaps tma_maps[2];
    bool dag_tma_ready = false;
    DagLists lists{};
    bool ishi_ready = false;  // the DAG is an Ishikawa chain: chain-specialised kernel
    TmaMaps ishi_maps[2];
    bool tree_ready = false;  // the DAG is a two-level tree: tree-specialised kernel
    TreeShape tree{};
    TmaMaps tree_maps[2];     // every node's flows (tree and four-inner-node kernels)
    bool dag4_ready = false;  // at most four non-end-label nodes: the four-inner-node kernel
    Dag4Shape dag4{};
    bool inplace_ready = false;
    InplaceMaps inplace_maps{};

    void set_data(const float* D, const float* S) override {
        base.D = D;
        base.S = S;
    }

    explicit Solver(const ProblemView& v) {
        base = make_step_args<MAXL, MAXN, IS_DAG>(v, 0);
        fused_smem = sizeof(float) * 3 * MAXL * FNE;
    }

    // TMA-staged in-place sweeps: Potts, NORMALISED (PAPER_LITERAL needs the
    // normaliser field between the sweeps and keeps the per-voxel kernels)
    bool inplace_tma() const { return kTmaCapable && inplace_ready && use_tma_inplace && !base.literal; }

    template <bool EXACT, bool IDX32>
    cudaError_t launch_inplace(const StepArgs<MAXL, MAXN>& a, dim3 grid, cudaStream_t s) {
        if constexpr (kTmaCapable) {
            using L = InplaceLayout<MAXL, DIM, T>;
            cudaError_t e = cudaFuncSetAttribute(prox_inplace_tma_kernel<MAXL, DIM, T, EXACT, IDX32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, L::p_total);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(flow_inplace_tma_kernel<MAXL, DIM, T, EXACT, IDX32>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, L::f_total);
            if (e != cudaSuccess) return e;
            prox_inplace_tma_kernel<MAXL, DIM, T, EXACT, IDX32><<<grid, INPLACE_TMA_NT, L::p_total, s>>>(a, inplace_maps);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            flow_inplace_tma_kernel<MAXL, DIM, T, EXACT, IDX32><<<grid, INPLACE_TMA_NT, L::f_total, s>>>(a, inplace_maps);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }

    template <bool WITH_E, bool IDX32>
    cudaError_t launch_ishikawa(const StepArgs<MAXL, MAXN>& a, const TmaMaps& m, dim3 grid, double* partial,
                                cudaStream_t s) {
        if constexpr (IS_DAG && DIM == 3) {
            using Lay = TmaLayout<ISH_MAXL, 3, T>;
            auto kern = ishikawa_tma_kernel<MAXL, MAXN, T, WITH_E, IDX32>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::total_bytes);
            if (e != cudaSuccess) return e;
            kern<<<grid, TMA_NT, Lay::total_bytes, s>>>(a, m, partial);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }

    template <bool IDX32, int G>
    cudaError_t launch_tree_g(const StepArgs<DMAX, DMAX>& a, const TmaMaps& m, dim3 grid, cudaStream_t s) {
        const TreeTmaLayout lay(a.nl, a.nn, DIM, (int)sizeof(T));
        cudaError_t e = cudaFuncSetAttribute(tree_tma_kernel<DIM, T, IDX32, G>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
        if (e != cudaSuccess) return e;
        tree_tma_kernel<DIM, T, IDX32, G><<<grid, DAG_TMA_NT, lay.total, s>>>(a, m, tree);
        return cudaGetLastError();
    }

    template <bool IDX32>
    cudaError_t launch_tree(const StepArgs<DMAX, DMAX>& a, const TmaMaps& m, dim3 grid, cudaStream_t s) {
        if constexpr (kDagTmaCapable) {
            // the kernel keeps per-group state in registers: compiled for 3 or 4 groups
            return tree.ng <= 3 ? launch_tree_g<IDX32, 3>(a, m, grid, s) : launch_tree_g<IDX32, 4>(a, m, grid, s);
        } else {
            return cudaErrorInvalidValue;
        }
    }

    template <bool IDX32>
    cudaError_t launch_dag4(const StepArgs<DMAX, DMAX>& a, const TmaMaps& m, dim3 grid, cudaStream_t s) {
        if constexpr (kDagTmaCapable) {
            const TreeTmaLayout lay(a.nl, a.nn, DIM, (int)sizeof(T));
            cudaError_t e = cudaFuncSetAttribute(dag4_tma_kernel<DIM, T, IDX32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
            if (e != cudaSuccess) return e;
            dag4_tma_kernel<DIM, T, IDX32><<<grid, DAG_TMA_NT, lay.total, s>>>(a, m, dag4);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }

    template <bool IDX32>
    cudaError_t launch_dag(const StepArgs<DMAX, DMAX>& a, const TmaMaps& m, dim3 grid, int smem, cudaStream_t s) {
        if constexpr (kDagTmaCapable) {
            cudaError_t e = cudaFuncSetAttribute(fused_dag_tma_kernel<DIM, T, IDX32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            fused_dag_tma_kernel<DIM, T, IDX32><<<grid, DAG_TMA_NT, smem, s>>>(a, m, lists);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }

    template <bool EXACT, bool WITH_E, bool IDX32>
    cudaError_t launch_tma3(const StepArgs<MAXL, MAXN>& a, const TmaMaps& m, dim3 grid, double* partial,
                            cudaStream_t s) {
        using Lay = TmaLayout<MAXL, DIM, T>;
        if constexpr (DIM == 3 && sizeof(T) == 2) {
            // 3-D, 16-bit storage: voxel pairs with packed FP32 arithmetic (the
            // one-voxel kernel is issue-bound there; with FP32 storage it is
            // at the bandwidth roof and the pair kernel measured slower); its
            // pair stores need an even row pitch
            if (a.px & 1) return cudaErrorInvalidValue;
            using XLay = X2Layout<MAXL, T>;
            cudaError_t e = cudaFuncSetAttribute(fused_tma_x2_kernel<MAXL, T, EXACT, WITH_E, IDX32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, XLay::total_bytes);
            if (e != cudaSuccess) return e;
            fused_tma_x2_kernel<MAXL, T, EXACT, WITH_E, IDX32><<<grid, X2_NT, XLay::total_bytes, s>>>(a, m, partial);
            return cudaGetLastError();
        } else {
            // the one-voxel kernel (not instantiated for 3-D 16-bit storage, which never runs it)
            cudaError_t e = cudaFuncSetAttribute(fused_tma_kernel<MAXL, DIM, T, EXACT, WITH_E, IDX32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::total_bytes);
            if (e != cudaSuccess) return e;
            fused_tma_kernel<MAXL, DIM, T, EXACT, WITH_E, IDX32><<<grid, TMA_NT, Lay::total_bytes, s>>>(a, m, partial);
            return cudaGetLastError();
        }
    }

    // 32-bit slot offsets when every offset of the flow array fits
    template <bool EXACT, bool WITH_E>
    cudaError_t launch_tma(const StepArgs<MAXL, MAXN>& a, const TmaMaps& m, dim3 grid, double* partial,
                           cudaStream_t s) {
        if ((long long)DIM * a.nn * a.n <= 0xFFFFFFFFll) return launch_tma3<EXACT, WITH_E, true>(a, m, grid, partial, s);
        return launch_tma3<EXACT, WITH_E, false>(a, m, grid, partial, s);
    }

    cudaError_t step(const void* u_in, void* u_out, const void* q_in, void* q_out, bool fused, int zc,
                     cudaStream_t s, int* launches, double* partial, int* nblocks) override {
        StepArgs<MAXL, MAXN> a = base;
        a.u_in = u_in;
        a.u_out = u_out;
        a.q_in = q_in;
        a.q_out = q_out;
        if (nblocks) *nblocks = 0;
        if constexpr (kTmaCapable) {
            if (fused && tma_ready && use_tma) {
                const int k = (u_in == tma_u[0]) ? 0 : 1;
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + FTY - 1) / FTY, (a.nz + a.zc - 1) / a.zc);
                const bool exact = a.nl == MAXL;
                cudaError_t e;
                if (partial) {
                    e = exact ? launch_tma<true, true>(a, tma_maps[k], grid, partial, s)
                              : launch_tma<false, true>(a, tma_maps[k], grid, partial, s);
                    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
                } else {
                    e = exact ? launch_tma<true, false>(a, tma_maps[k], grid, nullptr, s)
                              : launch_tma<false, false>(a, tma_maps[k], grid, nullptr, s);
                }
                *launches = 1;
                return e;
            }
        }
        if constexpr (IS_DAG && DIM == 3) {
            if (fused && ishi_ready && use_tma && use_ishi) {
                const int k = (u_in == tma_u[0]) ? 0 : 1;
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + FTY - 1) / FTY, (a.nz + a.zc - 1) / a.zc);
                *launches = 1;
                const bool idx32 = (long long)DIM * a.nn * a.n <= 0xFFFFFFFFll;
                if (partial) {
                    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
                    return idx32 ? launch_ishikawa<true, true>(a, ishi_maps[k], grid, partial, s)
                                 : launch_ishikawa<true, false>(a, ishi_maps[k], grid, partial, s);
                }
                return idx32 ? launch_ishikawa<false, true>(a, ishi_maps[k], grid, nullptr, s)
                             : launch_ishikawa<false, false>(a, ishi_maps[k], grid, nullptr, s);
            }
        }
        if constexpr (kDagTmaCapable) {
            if (fused && tree_ready && use_tma && use_tree) {
                const int k = (u_in == tma_u[0]) ? 0 : 1;
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + DTY - 1) / DTY, (a.nz + a.zc - 1) / a.zc);
                *launches = 1;
                const StepArgs<DMAX, DMAX> w = widen_args(a);
                if ((long long)DIM * a.nn * a.n <= 0xFFFFFFFFll) return launch_tree<true>(w, tree_maps[k], grid, s);
                return launch_tree<false>(w, tree_maps[k], grid, s);
            }
            if (fused && dag4_ready && use_tma && use_dag4) {
                const int k = (u_in == tma_u[0]) ? 0 : 1;
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + DTY - 1) / DTY, (a.nz + a.zc - 1) / a.zc);
                *launches = 1;
                const StepArgs<DMAX, DMAX> w = widen_args(a);
                if ((long long)DIM * a.nn * a.n <= 0xFFFFFFFFll) return launch_dag4<true>(w, tree_maps[k], grid, s);
                return launch_dag4<false>(w, tree_maps[k], grid, s);
            }
            if (fused && dag_tma_ready && use_tma) {
                const int k = (u_in == tma_u[0]) ? 0 : 1;
                a.zc = zc < 1 ? 1 : zc;
                const DagTmaLayout lay(a.nl, lists.nf, DIM, (int)sizeof(T));
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + DTY - 1) / DTY, (a.nz + a.zc - 1) / a.zc);
                *launches = 1;
                // 32-bit slot offsets when every offset of the flow array fits
                const StepArgs<DMAX, DMAX> w = widen_args(a);
                if ((long long)DIM * a.nn * a.n <= 0xFFFFFFFFll) return launch_dag<true>(w, tma_maps[k], grid, lay.total, s);
                return launch_dag<false>(w, tma_maps[k], grid, lay.total, s);
            }
        }
        if (fused) {
            if (fused_smem > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<MAXL, MAXN, DIM, IS_DAG, T>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)fused_smem);
                if (e != cudaSuccess) return e;
            }
            a.zc = zc < 1 ? 1 : zc;
            dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + FTY - 1) / FTY, (a.nz + a.zc - 1) / a.zc);
            fused_step_kernel<MAXL, MAXN, DIM, IS_DAG, T><<<grid, FUSED_NT, fused_smem, s>>>(a);
            *launches = 1;
        } else if (inplace_tma()) {
            if constexpr (kTmaCapable) {
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + FTY - 1) / FTY, (a.nz + a.zc - 1) / a.zc);
                *launches = 2;
                const bool exact = a.nl == MAXL;
                const bool idx32 = (long long)DIM * a.nn * a.n <= 0xFFFFFFFFll;
                if (exact) return idx32 ? launch_inplace<true, true>(a, grid, s) : launch_inplace<true, false>(a, grid, s);
                return idx32 ? launch_inplace<false, true>(a, grid, s) : launch_inplace<false, false>(a, grid, s);
            }
        } else {
            const unsigned blocks = (unsigned)((a.n + POINT_NT - 1) / POINT_NT);
            prox_inplace_kernel<MAXL, MAXN, DIM, IS_DAG, T><<<blocks, POINT_NT, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            flow_inplace_kernel<MAXL, MAXN, DIM, IS_DAG, T><<<blocks, POINT_NT, 0, s>>>(a);
            *launches = 2;
        }
        return cudaGetLastError();
    }

    // Maps of the chain-specialised Ishikawa kernel when the DAG is an
    // Ishikawa chain (3-D, any DAG bucket).
    void prepare_ishikawa(void* const* u, void* const* q, const float* D, const float* S) {
        if constexpr (IS_DAG && DIM == 3) {
            if (!is_ishikawa_chain(base)) return;
            const int es = (int)sizeof(T);
            bool ok = true;
            for (int k = 0; k < 2 && ok; ++k) {
                ok = encode_ishikawa_maps(base, es, u[k], q[k], D, S, &ishi_maps[k]);
                tma_u[k] = u[k];
            }
            ishi_ready = ok;
        }
    }

    bool prepare_tma(void* const* u, void* const* q, const float* D, const float* S) override {
        if constexpr (kDagTmaCapable) {
            const int es = (int)sizeof(T);
            const StepArgs<DMAX, DMAX> w = widen_args(base);
            DagTmaLayout lay(1, 1, DIM, es);
            if (!build_dag_lists(w, DIM, es, &lists, &lay)) return false;
            for (int k = 0; k < 2; ++k) {
                if (!encode_dag_maps(w, DIM, es, lists.nf, u[k], q[k], D, S, &tma_maps[k], lay.qbx)) return false;
                tma_u[k] = u[k];
            }
            dag_tma_ready = true;
            prepare_ishikawa(u, q, D, S);
            // two-level trees and DAGs with at most four inner nodes: maps over
            // every node's flows
            const bool is_tree = build_tree_shape(w, DIM, es, &tree);
            const bool is_dag4 = build_dag4_shape(w, DIM, es, &dag4);
            if (is_tree || is_dag4) {
                bool ok = true;
                const TreeTmaLayout tl(w.nl, w.nn, DIM, es);
                for (int k = 0; k < 2 && ok; ++k)
                    ok = encode_dag_maps(w, DIM, es, w.nn, u[k], q[k], D, S, &tree_maps[k], tl.qbx);
                tree_ready = ok && is_tree;
                dag4_ready = ok && is_dag4;
            }
            return false;  // the energy reduction keeps its own (non-TMA) kernel
        } else if constexpr (!kTmaCapable) {
            prepare_ishikawa(u, q, D, S);
            return false;
        } else {
            using Lay = TmaLayout<MAXL, DIM, T>;
            const int es = (int)sizeof(T);
            // every row pitch must be a multiple of 16 bytes (FP32 D and S too)
            if ((base.px * es) % 16 != 0 || (base.px * 4) % 16 != 0) return false;
            // logical extents, pitched strides: the padding is outside every box
            const unsigned long long nx = base.nx, ny = base.ny, nz = base.nz, nl = base.nl, px = base.px;
            const unsigned long long dims_u[4] = {nx, ny, nz, nl};
            const unsigned long long dims_q[4] = {nx, ny, nz, (unsigned long long)DIM * nl};
            const unsigned long long st_t[3] = {px * es, px * ny * es, px * ny * nz * es};
            const unsigned long long st_f[3] = {px * 4, px * ny * 4, px * ny * nz * 4};
            const unsigned box_u[4] = {(unsigned)TMA_BX, (unsigned)TMA_UY, 1u, (unsigned)nl};
            const unsigned box_q[4] = {(unsigned)Lay::QBX, (unsigned)TMA_QY, 1u, (unsigned)(DIM * nl)};
            const unsigned long long dims_s[3] = {nx, ny, nz};
            const unsigned box_s[3] = {(unsigned)FTX, (unsigned)FTY, 1u};
            for (int k = 0; k < 2; ++k) {
                TmaMaps& m = tma_maps[k];
                if (!encode_tiled_map(&m.u, u[k], es, 4, dims_u, st_t, box_u)) return false;
                if (!encode_tiled_map(&m.q, q[k], es, 4, dims_q, st_t, box_q)) return false;
                if (!encode_tiled_map(&m.D, D, 4, 4, dims_u, st_f, box_u)) return false;
                if (S) {
                    if (!encode_tiled_map(&m.S, S, 4, 3, dims_s, st_f, box_s)) return false;
                } else {
                    m.S = m.D;  // never read: the kernel skips S when the problem has no field
                }
                tma_u[k] = u[k];
            }
            tma_ready = true;
            // maps of the in-place sweeps (single buffer: u[0], q[0])
            {
                const unsigned box_t[4] = {(unsigned)FTX, (unsigned)FTY, 1u, (unsigned)nl};
                const unsigned box_qt[4] = {(unsigned)FTX, (unsigned)FTY, 1u, (unsigned)(DIM * nl)};
                InplaceMaps& im = inplace_maps;
                inplace_ready = encode_tiled_map(&im.u_tile, u[0], es, 4, dims_u, st_t, box_t) &&
                                encode_tiled_map(&im.D_tile, D, 4, 4, dims_u, st_f, box_t) &&
                                encode_tiled_map(&im.q_tile, q[0], es, 4, dims_q, st_t, box_qt);
                im.q_halo = tma_maps[0].q;
                im.u_halo = tma_maps[0].u;
                im.S = tma_maps[0].S;
            }
            return true;
        }
    }

    bool fuses_energy(bool fused) const override {
        return fused && use_tma && ((kTmaCapable && tma_ready) || (IS_DAG && ishi_ready && use_ishi));
    }

    void set_step(float c, float tau) override {
        base.inv_c = 1.0f / c;
        base.ctau = c * tau;
    }

    bool select(const char* name) override {
        const auto is = [&](const char* v) { return strcmp(name, v) == 0; };
        if (is("fused")) {
            use_tma = false;
            return true;
        }
        if (is("fused_tma") && kTmaCapable && tma_ready) {
            use_tma = true;
            return true;
        }
        if (is("fused_tma_ishikawa") && IS_DAG && ishi_ready) {
            use_tma = use_ishi = true;
            return true;
        }
        if (is("fused_tma_tree") && kDagTmaCapable && tree_ready) {
            use_tma = use_tree = true;
            use_ishi = false;
            return true;
        }
        if (is("fused_tma_dag4") && kDagTmaCapable && dag4_ready) {
            use_tma = use_dag4 = true;
            use_tree = use_ishi = false;
            return true;
        }
        if (is("fused_tma_dag") && kDagTmaCapable && dag_tma_ready) {
            use_tma = true;
            use_tree = use_ishi = use_dag4 = false;
            return true;
        }
        return false;
    }

    const char* variant(bool fused) const override {
        if (!fused) return inplace_tma() ? "inplace_tma" : "inplace";
        if (kTmaCapable && tma_ready && use_tma) return "fused_tma";
        if (IS_DAG && ishi_ready && use_tma && use_ishi) return "fused_tma_ishikawa";
        if (kDagTmaCapable && tree_ready && use_tma && use_tree) return "fused_tma_tree";
        if (kDagTmaCapable && dag4_ready && use_tma && use_dag4) return "fused_tma_dag4";
        if (kDagTmaCapable && dag_tma_ready && use_tma) return "fused_tma_dag";
        return "fused";
    }

    long long tma_energy_blocks(int zc) const override {
        // one partial per CTA of a TMA energy kernel or of an iteration that
        // reduces its input (Potts and Ishikawa kernels: 32 x 8 tiles; the
        // four-inner-node energy kernel: 32 x 4)
        zc = zc < 1 ? 1 : zc;
        const long long chunks = (base.nz + zc - 1) / zc, tx = (base.nx + FTX - 1) / FTX;
        long long nb = 0;
        if ((kTmaCapable && tma_ready) || (IS_DAG && ishi_ready)) nb = tx * ((base.ny + FTY - 1) / FTY) * chunks;
        if (IS_DAG && dag4_ready) nb = std::max(nb, tx * ((base.ny + DTY - 1) / DTY) * chunks);
        return nb;
    }

    cudaError_t energy(const void* u, const void* q, double* partial, int max_blocks, int zc, cudaStream_t s,
                       int* nblocks) override {
        StepArgs<MAXL, MAXN> a = base;
        a.u_in = u;
        a.q_in = q;
        if constexpr (kTmaCapable) {
            const long long nb = tma_energy_blocks(zc);
            if (nb > 0 && nb <= max_blocks) {
                using Lay = TmaLayout<MAXL, DIM, T>;
                const int k = (u == tma_u[0]) ? 0 : 1;
                cudaError_t e = cudaFuncSetAttribute(energy_tma_kernel<MAXL, DIM, T>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::total_bytes);
                if (e != cudaSuccess) return e;
                a.zc = zc < 1 ? 1 : zc;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + FTY - 1) / FTY, (a.nz + a.zc - 1) / a.zc);
                energy_tma_kernel<MAXL, DIM, T><<<grid, ENERGY_TMA_NT, Lay::total_bytes, s>>>(a, tma_maps[k], partial);
                *nblocks = (int)nb;
                return cudaGetLastError();
            }
        }
        if constexpr (kDagTmaCapable) {
            // DAGs with at most four inner nodes (HMF, DAGMF): the TMA energy
            // kernel in the four-inner-node layout, over the iteration's maps
            const int zcl = zc < 1 ? 1 : zc;
            const long long nb = (long long)((a.nx + FTX - 1) / FTX) * ((a.ny + DTY - 1) / DTY) *
                                 ((a.nz + zcl - 1) / zcl);
            if (dag4_ready && nb <= max_blocks) {
                StepArgs<DMAX, DMAX> w = widen_args(a);
                w.zc = zcl;
                const TreeTmaLayout lay(w.nl, w.nn, DIM, (int)sizeof(T));
                const int smem = lay.g_off + 64 + 128;  // the stages and their barriers
                const int k = (u == tma_u[0]) ? 0 : 1;
                cudaError_t e = cudaFuncSetAttribute(energy_dag4_tma_kernel<DIM, T>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                if (e != cudaSuccess) return e;
                dim3 grid((a.nx + FTX - 1) / FTX, (a.ny + DTY - 1) / DTY, (a.nz + zcl - 1) / zcl);
                energy_dag4_tma_kernel<DIM, T><<<grid, ENERGY4_NT, smem, s>>>(w, tree_maps[k], dag4, partial);
                *nblocks = (int)nb;
                return cudaGetLastError();
            }
        }
        const int blocks = (int)std::min<long long>((a.n + ENERGY_NT - 1) / ENERGY_NT, (long long)max_blocks);
        energy_partial_kernel<MAXL, MAXN, DIM, IS_DAG, T><<<blocks, ENERGY_NT, 0, s>>>(a, partial);
        *nblocks = blocks;
        return cudaGetLastError();
    }
};

// ---------------------------------------------------------------------------
// Batched iteration over many volumes (pfm_batch_*).
// ---------------------------------------------------------------------------
struct BatchMember {
    ProblemView view;
    void* u[2];
    void* q[2];
};

struct BatchBase {
    virtual ~BatchBase() {}
    // Builds the argument table (both parities) and the work list for chunk length zc.
    virtual cudaError_t setup(const BatchMember* m, int n, int zc) = 0;
    // One iteration of every member: inputs are buffer `parity`, outputs 1 - parity.
    virtual cudaError_t launch(int parity, int grid, cudaStream_t s) = 0;
    virtual int n_items() const = 0;
    // Resident CTAs per SM of the batched kernel (occupancy).
    virtual int ctas_per_sm() const = 0;
    // E and P of every member's state `parity` into energy_out()[2 k],
    // [2 k + 1] on the device: one launch over the batch's tiles and one
    // fixed-order reduction per member.  Runners without it return false
    // from has_energy (the members are then reduced one by one).
    virtual bool has_energy() const { return false; }
    virtual cudaError_t energy(int parity, cudaStream_t s) { return cudaErrorNotSupported; }
    virtual const double* energy_out() const { return nullptr; }
};

template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
struct BatchRunner final : BatchBase {
    using Args = StepArgs<MAXL, MAXN>;
    Args* dev = nullptr;   // [2][nvol]
    int4* items = nullptr;
    int nvol = 0, nitems = 0;
    size_t smem = batch_smem_bytes<MAXL, MAXN>();

    ~BatchRunner() override {
        if (dev) cudaFree(dev);
        if (items) cudaFree(items);
    }

    static Args make_args(const ProblemView& v, int zc) { return make_step_args<MAXL, MAXN, IS_DAG>(v, zc); }

    cudaError_t setup(const BatchMember* m, int n, int zc) override {
        if (dev) cudaFree(dev);
        if (items) cudaFree(items);
        dev = nullptr;
        items = nullptr;
        nvol = n;
        std::vector<Args> host(2 * (size_t)n);
        std::vector<int4> work;
        for (int k = 0; k < n; ++k) {
            for (int p = 0; p < 2; ++p) {
                Args a = make_args(m[k].view, zc);
                a.u_in = m[k].u[p];
                a.u_out = m[k].u[1 - p];
                a.q_in = m[k].q[p];
                a.q_out = m[k].q[1 - p];
                host[(size_t)p * n + k] = a;
            }
            const ProblemView& v = m[k].view;
            // x tiles fastest, so the CTAs that run together are neighbours
            for (int bz = 0; bz < (v.nz + zc - 1) / zc; ++bz)
                for (int by = 0; by < (v.ny + FTY - 1) / FTY; ++by)
                    for (int bx = 0; bx < (v.nx + FTX - 1) / FTX; ++bx) work.push_back(make_int4(k, bx, by, bz));
        }
        nitems = (int)work.size();
        cudaError_t e = cudaMalloc(&dev, sizeof(Args) * host.size());
        if (e != cudaSuccess) return e;
        e = cudaMalloc(&items, sizeof(int4) * work.size());
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(dev, host.data(), sizeof(Args) * host.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(items, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(batched_step_kernel<MAXL, MAXN, DIM, IS_DAG, T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }

    cudaError_t launch(int parity, int grid, cudaStream_t s) override {
        batched_step_kernel<MAXL, MAXN, DIM, IS_DAG, T>
            <<<grid, FUSED_NT, smem, s>>>(dev + (size_t)parity * nvol, items, nitems);
        return cudaGetLastError();
    }

    int n_items() const override { return nitems; }

    int ctas_per_sm() const override {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_step_kernel<MAXL, MAXN, DIM, IS_DAG, T>,
                                                          FUSED_NT, smem) != cudaSuccess)
            b = 1;
        cudaGetLastError();
        return b < 1 ? 1 : b;
    }
};

// Batched DAG iteration on the TMA-staged kernel: one persistent launch per
// iteration walks (member, x tile, y tile, z chunk) items; per member and
// parity the arguments and tensor maps sit in device memory, the lists once
// per member.
template <int DIM, typename T>
struct BatchDagTma final : BatchBase {
    using Args = StepArgs<DMAX, DMAX>;
    Args* args = nullptr;     // [2][nvol]
    TmaMaps* maps = nullptr;  // [2][nvol]
    DagLists* lists = nullptr;
    int4* items = nullptr;
    int* counter = nullptr;  // next work item of the running launch
    int nvol = 0, nitems = 0, smem = 0, bar_off = 0;
    bool idx32 = true;       // every member's slot offsets fit in 32 bits

    ~BatchDagTma() override { release(); }

    void release() {
        if (args) cudaFree(args);
        if (maps) cudaFree(maps);
        if (lists) cudaFree(lists);
        if (items) cudaFree(items);
        if (counter) cudaFree(counter);
        args = nullptr;
        maps = nullptr;
        lists = nullptr;
        items = nullptr;
        counter = nullptr;
    }

    // True if every member can run the TMA DAG kernel.
    static bool fits(const BatchMember* m, int n) {
        for (int k = 0; k < n; ++k) {
            if (m[k].view.nl > DMAX || m[k].view.nn > DMAX) return false;
            DagLists l;
            DagTmaLayout lay(1, 1, DIM, (int)sizeof(T));
            if (!build_dag_lists(make_step_args<DMAX, DMAX, true>(m[k].view, 1), DIM, (int)sizeof(T), &l, &lay))
                return false;
        }
        return true;
    }

    cudaError_t setup(const BatchMember* m, int n, int zc) override {
        release();
        nvol = n;
        const int es = (int)sizeof(T);
        std::vector<Args> ha(2 * (size_t)n);
        std::vector<TmaMaps> hm(2 * (size_t)n);
        std::vector<DagLists> hl((size_t)n);
        std::vector<int4> work;
        smem = 0;
        bar_off = 0;
        idx32 = true;
        for (int k = 0; k < n; ++k) {
            const ProblemView& v = m[k].view;
            idx32 = idx32 && (long long)DIM * v.nn * v.n <= 0xFFFFFFFFll;
            const Args base = make_step_args<DMAX, DMAX, true>(v, zc);
            DagTmaLayout lay(1, 1, DIM, es);
            if (!build_dag_lists(base, DIM, es, &hl[k], &lay)) return cudaErrorInvalidValue;
            smem = std::max(smem, lay.total);
            bar_off = std::max(bar_off, lay.bar_off);
            for (int p = 0; p < 2; ++p) {
                Args a = base;
                a.u_in = m[k].u[p];
                a.u_out = m[k].u[1 - p];
                a.q_in = m[k].q[p];
                a.q_out = m[k].q[1 - p];
                ha[(size_t)p * n + k] = a;
                if (!encode_dag_maps(base, DIM, es, hl[k].nf, m[k].u[p], m[k].q[p], v.D, v.S, &hm[(size_t)p * n + k],
                                     lay.qbx))
                    return cudaErrorInvalidValue;
            }
            // x tiles fastest, so the CTAs that run together are neighbours
            for (int bz = 0; bz < (v.nz + zc - 1) / zc; ++bz)
                for (int by = 0; by < (v.ny + DTY - 1) / DTY; ++by)
                    for (int bx = 0; bx < (v.nx + FTX - 1) / FTX; ++bx) work.push_back(make_int4(k, bx, by, bz));
        }
        // the barriers sit past every member's buffers; + 64 bytes for them
        smem = std::max(smem, bar_off + 64 + 128);
        nitems = (int)work.size();
        cudaError_t e;
        if ((e = cudaMalloc(&args, sizeof(Args) * ha.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&maps, sizeof(TmaMaps) * hm.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&lists, sizeof(DagLists) * hl.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&items, sizeof(int4) * work.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&counter, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(args, ha.data(), sizeof(Args) * ha.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(maps, hm.data(), sizeof(TmaMaps) * hm.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(lists, hl.data(), sizeof(DagLists) * hl.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(items, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(batched_dag_tma_kernel<DIM, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem)) != cudaSuccess)
            return e;
        return cudaFuncSetAttribute(batched_dag_tma_kernel<DIM, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem);
    }

    cudaError_t launch(int parity, int grid, cudaStream_t s) override {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (idx32)
            batched_dag_tma_kernel<DIM, T, true><<<grid, DAG_TMA_NT, smem, s>>>(
                args + (size_t)parity * nvol, maps + (size_t)parity * nvol, lists, items, nitems, bar_off, counter);
        else
            batched_dag_tma_kernel<DIM, T, false><<<grid, DAG_TMA_NT, smem, s>>>(
                args + (size_t)parity * nvol, maps + (size_t)parity * nvol, lists, items, nitems, bar_off, counter);
        return cudaGetLastError();
    }

    int n_items() const override { return nitems; }
    int ctas_per_sm() const override { return 1; }
};

// Batched iteration on the four-inner-node kernel (every member a DAG with
// at most four non-end-label nodes and twelve end-labels): one persistent
// launch per iteration over (member, x tile, y tile, z chunk) items; per
// member and parity the arguments and tensor maps (every node's flows) in
// device memory, the shapes once per member.
template <int DIM, typename T>
struct BatchDag4Tma final : BatchBase {
    using Args = StepArgs<DMAX, DMAX>;
    Args* args = nullptr;       // [2][nvol]
    TmaMaps* maps = nullptr;    // [2][nvol]
    Dag4Shape* shapes = nullptr;
    int4* items = nullptr;
    int* counter = nullptr;     // next work item of the running launch
    int* ebegin = nullptr;      // [nvol + 1]: each member's first work item
    double* epartial = nullptr; // [nitems][2]: (E, P) of every work item
    double* eout = nullptr;     // [nvol][2]
    int nvol = 0, nitems = 0, smem = 0, bar_off = 0, esmem = 0;
    bool idx32 = true;

    ~BatchDag4Tma() override { release(); }

    void release() {
        void* ptrs[] = {args, maps, shapes, items, counter, ebegin, epartial, eout};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        args = nullptr;
        maps = nullptr;
        shapes = nullptr;
        items = nullptr;
        counter = nullptr;
        ebegin = nullptr;
        epartial = nullptr;
        eout = nullptr;
    }

    bool has_energy() const override { return true; }
    const double* energy_out() const override { return eout; }
    cudaError_t energy(int parity, cudaStream_t s) override {
        batched_energy_dag4_tma_kernel<DIM, T><<<nitems, ENERGY4_NT, esmem, s>>>(
            args + (size_t)parity * nvol, maps + (size_t)parity * nvol, shapes, items, epartial);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        energy_final_ranges_kernel<<<nvol, ENERGY_RANGES_NT, 0, s>>>(epartial, ebegin, args + (size_t)parity * nvol,
                                                                       eout);
        return cudaGetLastError();
    }

    // True if every member can run the four-inner-node kernel.
    static bool fits(const BatchMember* m, int n) {
        for (int k = 0; k < n; ++k) {
            if (m[k].view.nl > DMAX || m[k].view.nn > DMAX) return false;
            Dag4Shape sh;
            if (!build_dag4_shape(make_step_args<DMAX, DMAX, true>(m[k].view, 1), DIM, (int)sizeof(T), &sh))
                return false;
        }
        return true;
    }

    cudaError_t setup(const BatchMember* m, int n, int zc) override {
        release();
        nvol = n;
        const int es = (int)sizeof(T);
        std::vector<Args> ha(2 * (size_t)n);
        std::vector<TmaMaps> hm(2 * (size_t)n);
        std::vector<Dag4Shape> hs((size_t)n);
        std::vector<int4> work;
        smem = 0;
        bar_off = 0;
        esmem = 0;
        idx32 = true;
        std::vector<int> begin((size_t)n + 1, 0);
        for (int k = 0; k < n; ++k) {
            const ProblemView& v = m[k].view;
            idx32 = idx32 && (long long)DIM * v.nn * v.n <= 0xFFFFFFFFll;
            const Args base = make_step_args<DMAX, DMAX, true>(v, zc);
            if (!build_dag4_shape(base, DIM, es, &hs[k])) return cudaErrorInvalidValue;
            const TreeTmaLayout lay(v.nl, v.nn, DIM, es);
            smem = std::max(smem, lay.total);
            bar_off = std::max(bar_off, lay.bar_off);
            esmem = std::max(esmem, lay.g_off + 64 + 128);  // the energy kernel: stages and barriers
            begin[k] = (int)work.size();
            for (int p = 0; p < 2; ++p) {
                Args a = base;
                a.u_in = m[k].u[p];
                a.u_out = m[k].u[1 - p];
                a.q_in = m[k].q[p];
                a.q_out = m[k].q[1 - p];
                ha[(size_t)p * n + k] = a;
                if (!encode_dag_maps(base, DIM, es, v.nn, m[k].u[p], m[k].q[p], v.D, v.S, &hm[(size_t)p * n + k],
                                     lay.qbx))
                    return cudaErrorInvalidValue;
            }
            // x tiles fastest, so the CTAs that run together are neighbours
            for (int bz = 0; bz < (v.nz + zc - 1) / zc; ++bz)
                for (int by = 0; by < (v.ny + DTY - 1) / DTY; ++by)
                    for (int bx = 0; bx < (v.nx + FTX - 1) / FTX; ++bx) work.push_back(make_int4(k, bx, by, bz));
        }
        // the barriers sit past every member's buffers
        smem = std::max(smem, bar_off + 64 + 128);
        nitems = (int)work.size();
        begin[n] = nitems;
        cudaError_t e;
        if ((e = cudaMalloc(&ebegin, sizeof(int) * begin.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&epartial, sizeof(double) * 2 * (size_t)nitems)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&eout, sizeof(double) * 2 * (size_t)n)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(ebegin, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(batched_energy_dag4_tma_kernel<DIM, T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, esmem)) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(&args, sizeof(Args) * ha.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&maps, sizeof(TmaMaps) * hm.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&shapes, sizeof(Dag4Shape) * hs.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&items, sizeof(int4) * work.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&counter, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(args, ha.data(), sizeof(Args) * ha.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(maps, hm.data(), sizeof(TmaMaps) * hm.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(shapes, hs.data(), sizeof(Dag4Shape) * hs.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(items, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(batched_dag4_tma_kernel<DIM, T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        return cudaFuncSetAttribute(batched_dag4_tma_kernel<DIM, T, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }

    cudaError_t launch(int parity, int grid, cudaStream_t s) override {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (idx32)
            batched_dag4_tma_kernel<DIM, T, true><<<grid, DAG_TMA_NT, smem, s>>>(
                args + (size_t)parity * nvol, maps + (size_t)parity * nvol, shapes, items, nitems, bar_off, counter);
        else
            batched_dag4_tma_kernel<DIM, T, false><<<grid, DAG_TMA_NT, smem, s>>>(
                args + (size_t)parity * nvol, maps + (size_t)parity * nvol, shapes, items, nitems, bar_off, counter);
        return cudaGetLastError();
    }

    int n_items() const override { return nitems; }
    int ctas_per_sm() const override { return 1; }
};

// Factories, one per translation unit (storage x model).
SolverBase* make_potts_f32(int maxl, int dim, const ProblemView& v);
SolverBase* make_potts_bf16(int maxl, int dim, const ProblemView& v);
SolverBase* make_potts_f16(int maxl, int dim, const ProblemView& v);
SolverBase* make_dag_f32(int maxl, int maxn, int dim, const ProblemView& v);
SolverBase* make_dag_bf16(int maxl, int maxn, int dim, const ProblemView& v);
SolverBase* make_dag_f16(int maxl, int maxn, int dim, const ProblemView& v);
BatchBase* make_batch_potts_f32(int maxl, int dim);
BatchBase* make_batch_potts_bf16(int maxl, int dim);
BatchBase* make_batch_potts_f16(int maxl, int dim);
BatchBase* make_batch_dag_f32(int maxl, int maxn, int dim);
BatchBase* make_batch_dag_bf16(int maxl, int maxn, int dim);
BatchBase* make_batch_dag_f16(int maxl, int maxn, int dim);
// The TMA DAG batch, or nullptr if some member cannot run the TMA DAG kernel.
BatchBase* make_batch_dag_tma_f32(const BatchMember* m, int n, int dim);
BatchBase* make_batch_dag_tma_bf16(const BatchMember* m, int n, int dim);
BatchBase* make_batch_dag_tma_f16(const BatchMember* m, int n, int dim);
// The four-inner-node batch, or nullptr if some member cannot run that kernel.
BatchBase* make_batch_dag4_tma_f32(const BatchMember* m, int n, int dim);
BatchBase* make_batch_dag4_tma_bf16(const BatchMember* m, int n, int dim);
BatchBase* make_batch_dag4_tma_f16(const BatchMember* m, int n, int dim);

// Adjoint of one Potts iteration (pfm_adjoint.cu).
struct AdjLaunch {
    const float* u_k;      // [nl][n]
    const float* q_k;      // [nl][dim][n]
    const float* u_k1;     // [nl][n]
    const float* ubar_k1;  // [nl][n]
    const float* qbar_k1;  // [nl][dim][n]
    float* ubar_k;         // [nl][n]  (may alias ubar_k1)
    float* qbar_k;         // [nl][dim][n]  (may alias qbar_k1)
    float* Dbar;           // [nl][n], accumulated
    float* Sbar;           // [n], accumulated, or nullptr
    float* ybar;           // work [nl][dim][n]
    float* dbar;           // work [nl][n]
    const float* D;        // the problem's [nl][np], rows of pitch px
    const float* S;        // the problem's [np], or nullptr
    int nx, ny, nz, nl;
    int px;                // row pitch of D and S
    long long n;           // dense voxels of the caller's arrays
    long long np;          // slots per label of D (px*ny*nz)
    float c, ctau;
    int aniso;
    float s_node[16];
};
cudaError_t launch_adjoint(const AdjLaunch& a, int ndim, cudaStream_t s);

// Explicit-flow augmented-Lagrangian solver (pfm_alm.cu).
struct AlmArgs {
    float* u;      // [nl][n] multipliers (the labelling)
    float* q;      // [nl][dim][n]
    float* pL;     // [nl][n] sink flows
    float* pS;     // [n] source flow
    float* f;      // [nl][n] work
    const float* D;
    const float* S;
    int nx, ny, nz, nl;
    long long n;
    float gamma, step;
    int aniso;
    float s_node[16];
};
cudaError_t launch_alm_init(const AlmArgs& a, cudaStream_t s);
cudaError_t launch_alm_iteration(const AlmArgs& a, int ndim, cudaStream_t s);
cudaError_t launch_sum(const float* v, long long n, double* partial, int blocks, cudaStream_t s);

// Auxiliary kernels (pfm_misc.cu).
cudaError_t launch_init_labels(void* u, int storage, int nl, long long n, cudaStream_t s);
// Readback and import between the pitched internal arrays (rows of nx
// values at pitch px, n = px*ny*nz slots per label) and dense caller arrays.
cudaError_t launch_argmax(const void* u, int storage, int nl, long long n, int nx, int px, long long nv, int* out,
                          cudaStream_t s);
cudaError_t launch_to_f32(const void* src, int storage, long long rows, int nx, int px, float* dst, cudaStream_t s);
cudaError_t launch_set_labels(const float* src, int storage, int nl, long long nv, int nx, int px, long long n,
                              void* dst, unsigned* flags, cudaStream_t s);
cudaError_t launch_set_flows(const float* src, int storage, int nn, int ndim, int nx, int ny, int nz, int px,
                             const float* s_node_dev, const float* S, int aniso, void* dst, cudaStream_t s);
// ORs *src into *dst (one thread).
cudaError_t launch_merge_flags(const unsigned* src, unsigned* dst, cudaStream_t s);
cudaError_t launch_validate(const float* D, long long nD, const float* S, long long nS, unsigned* flags,
                            cudaStream_t s);
cudaError_t launch_energy_final(const double* partial, int blocks, double* out, unsigned* flags, cudaStream_t s);

}  // namespace pfm
