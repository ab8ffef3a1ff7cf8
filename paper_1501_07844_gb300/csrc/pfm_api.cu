// pfm_api.cu -- the C ABI of libpfm (declared in include/pfm.h).
//
// Owns device state, validates problems (the label DAG of Section 3.3 and
// the data), picks a kernel bucket, and queues iterations, energy/gap
// reductions and readbacks on the problem's CUDA stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <string>
#include <vector>

#include "../../include/pfm.h"
#include "pfm_solver.cuh"

namespace {

thread_local std::string g_err;

pfm_status fail(pfm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

pfm_status cuda_fail(cudaError_t e, const char* where) {
    const pfm_status st = (e == cudaErrorMemoryAllocation) ? PFM_ENOMEM : PFM_ECUDA;
    return fail(st, "%s: %s", where, cudaGetErrorString(e));
}

#define PFM_CUDA(call, where)                         \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// Validated, host-side description of a label DAG.
struct DagInfo {
    int nn = 0, nl = 0;
    bool flat = false;               // the Potts model: S -> every node, w = 1
    std::vector<int> leaf_node;      // end-label j -> node id (ascending)
    std::vector<double> W;           // [nn][nn] path weights W_(A,B)
};

// Checks the DAG of a problem description and computes path weights
// W_(A,B) (Section 3.3 recursion) and the end-label list.
pfm_status analyse_dag(const pfm_desc* d, DagInfo* out) {
    const int nn = d->n_nodes, ne = d->n_edges;
    if (nn < 1 || ne < 1 || !d->edge_parent || !d->edge_child || !d->edge_w)
        return fail(PFM_EDAG, "DAG needs n_nodes >= 1 and n_edges >= 1 with edge arrays");
    std::vector<int> indeg(nn, 0), nchild(nn, 0), rem(nn, 0);
    for (int e = 0; e < ne; ++e) {
        const int a = d->edge_parent[e], b = d->edge_child[e];
        const double w = d->edge_w[e];
        if (a < -1 || a >= nn || b < 0 || b >= nn || a == b)
            return fail(PFM_EDAG, "edge %d (%d -> %d) out of range or self loop", e, a, b);
        if (!(w > 0.0) || !isfinite(w)) return fail(PFM_EDAG, "edge %d weight must be finite and > 0", e);
        indeg[b]++;
        if (a >= 0) {
            nchild[a]++;
            rem[b]++;
        }
    }
    for (int v = 0; v < nn; ++v)
        if (indeg[v] == 0) return fail(PFM_EDAG, "node %d has no parent (unreachable from the source)", v);
    // topological order (Kahn), source edges satisfied from the start
    std::vector<int> order;
    order.reserve(nn);
    for (int v = 0; v < nn; ++v)
        if (rem[v] == 0) order.push_back(v);
    for (size_t h = 0; h < order.size(); ++h) {
        const int v = order[h];
        for (int e = 0; e < ne; ++e)
            if (d->edge_parent[e] == v && --rem[d->edge_child[e]] == 0) order.push_back(d->edge_child[e]);
    }
    if ((int)order.size() != nn) return fail(PFM_EDAG, "label graph has a cycle");
    out->nn = nn;
    out->leaf_node.clear();
    for (int v = 0; v < nn; ++v)
        if (nchild[v] == 0) out->leaf_node.push_back(v);
    out->nl = (int)out->leaf_node.size();
    out->W.assign((size_t)nn * nn, 0.0);
    for (int k = nn - 1; k >= 0; --k) {
        const int A = order[k];
        out->W[(size_t)A * nn + A] = 1.0;
        for (int e = 0; e < ne; ++e)
            if (d->edge_parent[e] == A)
                for (int B = 0; B < nn; ++B)
                    out->W[(size_t)A * nn + B] += d->edge_w[e] * out->W[(size_t)d->edge_child[e] * nn + B];
    }
    // W_(S,L) = 1 for every end-label: sum_L u_L = 1 is then u_S = 1
    for (int L : out->leaf_node) {
        double ws = 0.0;
        for (int e = 0; e < ne; ++e)
            if (d->edge_parent[e] == -1) ws += d->edge_w[e] * out->W[(size_t)d->edge_child[e] * nn + L];
        if (fabs(ws - 1.0) > 1e-9)
            return fail(PFM_EDAG, "end-label %d has source path weight %.12g (must be 1)", L, ws);
    }
    out->flat = (ne == nn);
    for (int e = 0; e < ne && out->flat; ++e)
        out->flat = d->edge_parent[e] == -1 && d->edge_w[e] == 1.0;
    return PFM_OK;
}

int potts_bucket(int nl) { return nl <= 4 ? 4 : nl <= 8 ? 8 : nl <= 16 ? 16 : 0; }

// z-chunk length of the plane-marching kernels from a cost model: a CTA of
// chunk length zc costs about zc + 3 plane times (the chunk, the flows of
// plane z0-1 and the pipeline fill), CTAs run in waves of `sms` (one CTA per
// SM: the staging ring takes most of the shared memory), so the launch
// costs ceil(CTAs / sms) * (zc + 3).  The chunk counts considered keep every
// SM busy in the first wave when the volume allows it.
int model_zc(long long tiles, int nz, int sms) {
    if (nz <= 4) return std::max(nz, 1);
    sms = std::max(sms, 1);
    long long best_cost = -1;
    int best = 4;
    const bool can_fill = tiles * ((nz + 3) / 4) >= sms;
    for (int c = 1; c <= nz; ++c) {
        const int zc = (nz + c - 1) / c;
        if (zc < 4) break;
        if (c > 1 && zc == (nz + c - 2) / (c - 1)) continue;  // same chunk length as c - 1
        const long long ctas = tiles * c;
        if (can_fill && ctas < sms) continue;
        const long long cost = ((ctas + sms - 1) / sms) * (zc + 3);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

int device_sms() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

long long zc_tiles(const pfm_problem* pb);
void dag_bucket(int nl, int nn, int* ml, int* mn) {
    *ml = *mn = 0;
    if (nl <= 8 && nn <= 12) {
        *ml = 8;
        *mn = 12;
    } else if (nl <= 16 && nn <= 16) {
        *ml = 16;
        *mn = 16;
    }
}

pfm_status check_params(const pfm_params* p) {
    if (!p) return fail(PFM_EINVAL, "params is NULL");
    if (!(p->c > 0) || !isfinite(p->c)) return fail(PFM_EINVAL, "c must be finite and > 0");
    if (!(p->tau > 0) || !isfinite(p->tau)) return fail(PFM_EINVAL, "tau must be finite and > 0");
    if (p->norm != PFM_NORM_ISO && p->norm != PFM_NORM_ANISO) return fail(PFM_EINVAL, "bad norm");
    if (p->grad_source != PFM_GRAD_NORMALISED && p->grad_source != PFM_GRAD_PAPER_LITERAL)
        return fail(PFM_EINVAL, "bad grad_source");
    if (p->storage != PFM_STORAGE_F32 && p->storage != PFM_STORAGE_BF16 && p->storage != PFM_STORAGE_F16)
        return fail(PFM_EINVAL, "bad storage");
    if (p->schedule != PFM_SCHEDULE_FUSED && p->schedule != PFM_SCHEDULE_INPLACE &&
        p->schedule != PFM_SCHEDULE_FUSED_PLAIN)
        return fail(PFM_EINVAL, "bad schedule");
    if (p->check_every < 1) return fail(PFM_EINVAL, "check_every must be >= 1");
    return PFM_OK;
}

pfm_status check_desc(const pfm_desc* d, DagInfo* dag) {
    if (!d) return fail(PFM_EINVAL, "desc is NULL");
    if (d->ndim != 2 && d->ndim != 3) return fail(PFM_EINVAL, "ndim must be 2 or 3");
    for (int k = 0; k < 3; ++k)
        if (d->dims[k] < 1 || d->dims[k] > (1 << 30)) return fail(PFM_EINVAL, "dims[%d] out of range", k);
    if (d->ndim == 2 && d->dims[2] != 1) return fail(PFM_EINVAL, "2-D problems need dims[2] == 1");
    const long long n = (long long)d->dims[0] * d->dims[1] * d->dims[2];
    if (n > (1ll << 40)) return fail(PFM_EINVAL, "grid too large");
    if (!d->D) return fail(PFM_EINVAL, "D is NULL");
    pfm_status st = analyse_dag(d, dag);
    if (st != PFM_OK) return st;
    if (d->s_node)
        for (int A = 0; A < d->n_nodes; ++A)
            if (!(d->s_node[A] >= 0.f) || !isfinite(d->s_node[A]))
                return fail(PFM_EINVAL, "s_node[%d] must be finite and >= 0", A);
    if (dag->flat) {
        if (!potts_bucket(dag->nl)) return fail(PFM_EUNSUPPORTED, "Potts supports at most 16 labels");
    } else {
        int ml, mn;
        dag_bucket(dag->nl, dag->nn, &ml, &mn);
        if (!ml) return fail(PFM_EUNSUPPORTED, "DAG models support at most 16 end-labels and 16 nodes");
    }
    return PFM_OK;
}

size_t elem_size(int storage) { return storage == PFM_STORAGE_F32 ? 4 : 2; }

}  // namespace

namespace pfm {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_tiled_map(CUtensorMap* map, const void* base, int elem_bytes, int rank, const unsigned long long* dims,
                      const unsigned long long* strides, const unsigned* box) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            return false;
        }
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    cuuint64_t d[5], s[4];
    cuuint32_t b[5], e[5];
    for (int k = 0; k < rank; ++k) {
        d[k] = dims[k];
        b[k] = box[k];
        e[k] = 1;
    }
    for (int k = 0; k + 1 < rank; ++k) s[k] = strides[k];
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // zero fill of out-of-bounds elements is the zero boundary flow
    return fn(map, dt, (cuuint32_t)rank, const_cast<void*>(base), d, s, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Sets the thread-local message returned by pfm_last_error (for entry points
// defined in other translation units).
pfm_status set_error(pfm_status st, const char* msg) {
    g_err = msg;
    return st;
}
}  // namespace pfm

struct pfm_problem {
    int ndim = 0, nx = 0, ny = 0, nz = 0, nl = 0, nn = 0;
    int px = 0;         // row pitch (elements) of every device array, >= nx
    long long n = 0;    // slots per label / component: px*ny*nz
    long long nv = 0;   // voxels: nx*ny*nz (the caller's dense arrays)
    bool flat = true;
    pfm_params prm{};
    cudaStream_t stream = nullptr;
    void* u[2] = {nullptr, nullptr};
    void* q[2] = {nullptr, nullptr};
    int cur = 0;
    float* D = nullptr;
    float* S = nullptr;
    float* abuf = nullptr;
    float* snode_dev = nullptr;
    unsigned* flags = nullptr;
    double* partial = nullptr;
    double* result = nullptr;
    int energy_blocks = 0;
    int zc = 32;
    std::vector<float> s_node;
    std::vector<float> W;  // [nn][nl]
    int64_t iters = 0, launches = 0;
    pfm::SolverBase* solver = nullptr;
    // double-buffered upload (pfm_prefetch_data / pfm_commit_data): the
    // staging buffers and D / S trade places at a commit (batch members, whose
    // buffers the batch's kernel arguments hold, copy instead)
    float* D_stage = nullptr;
    float* S_stage = nullptr;
    unsigned* stage_flags = nullptr;  // validation of the staged data
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t staged = nullptr;    // the prefetch copy is complete
    cudaEvent_t consumed = nullptr;  // work enqueued before the last commit (readers of the staging buffers) is done
    bool stage_pending = false;
    bool in_batch = false;
    // asynchronous argmax read-back (pfm_get_argmax_async)
    int* am_buf = nullptr;
    cudaEvent_t am_ready = nullptr;   // the argmax kernel has written am_buf
    cudaEvent_t am_done = nullptr;    // the copy out of am_buf has landed
};

namespace pfm {
// The reverse-mode steps of n consecutive iterations (pfm_adjoint.cu).
cudaError_t launch_adjoint_chain(const AdjLaunch* steps, int nsteps, int ndim, cudaStream_t s);
// A bounded mbarrier wait that nothing completes (pfm_misc.cu).
cudaError_t launch_wait_selftest(unsigned* flags, cudaStream_t s);
}  // namespace pfm

namespace {

// tiles of one z-chunk row of the grid: 32 x 4 for the TMA DAG kernel,
// 32 x 8 for every other kernel
long long zc_tiles(const pfm_problem* pb) {
    const char* v = pb->solver->variant(pb->prm.schedule != PFM_SCHEDULE_INPLACE);
    const int ty = (strcmp(v, "fused_tma_dag") == 0 || strcmp(v, "fused_tma_tree") == 0 ||
                    strcmp(v, "fused_tma_dag4") == 0)
                       ? pfm::DTY
                       : pfm::FTY;
    return (long long)((pb->nx + pfm::FTX - 1) / pfm::FTX) * ((pb->ny + ty - 1) / ty);
}

pfm::ProblemView view_of(const pfm_problem* pb) {
    pfm::ProblemView v{};
    v.ndim = pb->ndim;
    v.nx = pb->nx;
    v.px = pb->px;
    v.ny = pb->ny;
    v.nz = pb->nz;
    v.nl = pb->nl;
    v.nn = pb->nn;
    v.n = pb->n;
    v.c = (float)pb->prm.c;
    v.tau = (float)pb->prm.tau;
    v.literal = pb->prm.grad_source == PFM_GRAD_PAPER_LITERAL;
    v.aniso = pb->prm.norm == PFM_NORM_ANISO;
    v.D = pb->D;
    v.S = pb->S;
    v.abuf = pb->abuf;
    v.flags = pb->flags;
    v.s_node = pb->s_node.data();
    v.W = pb->W.data();
    return v;
}

pfm_status read_flags(pfm_problem* pb, unsigned* out) {
    unsigned h = 0;
    PFM_CUDA(cudaMemcpyAsync(&h, pb->flags, sizeof h, cudaMemcpyDeviceToHost, pb->stream), "read flags");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    *out = h;
    return PFM_OK;
}

pfm_status flags_status(unsigned f) {
    if (f & pfm::FLAG_TIMEOUT) return fail(PFM_ETIMEOUT, "a bounded device-side wait expired (TMA pipeline)");
    if (f & pfm::FLAG_BAD_INPUT) return fail(PFM_ENONFINITE, "D not finite or S negative / not finite");
    if (f & pfm::FLAG_NONFINITE) return fail(PFM_ENONFINITE, "non-finite normaliser, energy or dual");
    if (f & pfm::FLAG_BAD_LABELS) return fail(PFM_EINVAL, "labelling with a negative entry or zero sum");
    return PFM_OK;
}

void free_all(pfm_problem* pb) {
    // the in-place schedule aliases u[1] = u[0] and q[1] = q[0]
    if (pb->copy_stream) cudaStreamSynchronize(pb->copy_stream);
    void* ptrs[] = {pb->u[0], pb->u[1] != pb->u[0] ? pb->u[1] : nullptr, pb->q[0],
                    pb->q[1] != pb->q[0] ? pb->q[1] : nullptr, pb->D, pb->S, pb->abuf, pb->snode_dev,
                    pb->flags, pb->partial, pb->result, pb->D_stage, pb->S_stage, pb->stage_flags};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (pb->am_done) cudaEventSynchronize(pb->am_done);
    if (pb->am_buf) cudaFree(pb->am_buf);
    if (pb->am_ready) cudaEventDestroy(pb->am_ready);
    if (pb->am_done) cudaEventDestroy(pb->am_done);
    if (pb->staged) cudaEventDestroy(pb->staged);
    if (pb->consumed) cudaEventDestroy(pb->consumed);
    if (pb->copy_stream) cudaStreamDestroy(pb->copy_stream);
    cudaGetLastError();  // leave no stale error for the next call of this thread
    delete pb->solver;
    pb->solver = nullptr;
}

}  // namespace

extern "C" {

int pfm_version(void) { return PFM_VERSION; }

const char* pfm_last_error(void) { return g_err.c_str(); }

void pfm_params_default(pfm_params* p) {
    if (!p) return;
    p->c = 0.5;
    p->tau = 0.11;
    p->norm = PFM_NORM_ISO;
    p->grad_source = PFM_GRAD_NORMALISED;
    p->storage = PFM_STORAGE_F32;
    p->schedule = PFM_SCHEDULE_FUSED;
    p->check_every = 10;
    p->gap_tol = 1e-4;
}

}  // extern "C"

// Device arrays of pfm_create's problems have rows padded to a multiple of
// 8 elements (16 bytes in FP32 and BF16); the explicit-flow solver's are dense.
static pfm_status footprint_impl(const pfm_desc* desc, const pfm_params* params, bool dense, size_t* device_bytes,
                                 int64_t* n_grid_buffers, int* n_leaf_out) {
    DagInfo dag;
    pfm_status st = check_params(params);
    if (st != PFM_OK) return st;
    st = check_desc(desc, &dag);
    if (st != PFM_OK) return st;
    const long long px = dense ? desc->dims[0] : (desc->dims[0] + 7) / 8 * 8;
    const long long n = px * desc->dims[1] * desc->dims[2];
    const int copies = params->schedule == PFM_SCHEDULE_INPLACE ? 1 : 2;
    const size_t ts = elem_size(params->storage);
    int64_t bufs = 0;
    size_t bytes = 0;
    bufs += (int64_t)copies * dag.nl;                       // u
    bytes += (size_t)copies * dag.nl * n * ts;
    bufs += (int64_t)copies * dag.nn * desc->ndim;          // q
    bytes += (size_t)copies * dag.nn * desc->ndim * n * ts;
    bufs += dag.nl;                                          // D
    bytes += (size_t)dag.nl * n * 4;
    if (desc->S_field) {
        bufs += 1;
        bytes += (size_t)n * 4;
    }
    if (params->schedule == PFM_SCHEDULE_INPLACE && params->grad_source == PFM_GRAD_PAPER_LITERAL) {
        bufs += 1;                                           // accumulator a(x)
        bytes += (size_t)n * 4;
    }
    if (device_bytes) *device_bytes = bytes;
    if (n_grid_buffers) *n_grid_buffers = bufs;
    if (n_leaf_out) *n_leaf_out = dag.nl;
    return PFM_OK;
}

extern "C" {

pfm_status pfm_footprint(const pfm_desc* desc, const pfm_params* params, size_t* device_bytes,
                         int64_t* n_grid_buffers, int* n_leaf_out) {
    return footprint_impl(desc, params, false, device_bytes, n_grid_buffers, n_leaf_out);
}

// Row pitch of the device arrays: nx rounded up to 8 elements, so that every
// row of the FP32 and BF16 arrays starts on a 16-byte boundary (the TMA
// kernels need it); the explicit-flow solver keeps dense rows.
static int row_pitch(long long nx, bool dense) { return (int)(dense ? nx : (nx + 7) / 8 * 8); }

// Copy rows of nx FP32 values between a dense caller array and a pitched
// device array (either direction; pitches in elements).
static cudaError_t copy_rows(void* dst, int dpitch, const void* src, int spitch, int nx, long long rows,
                             cudaStream_t s) {
    if (dpitch == nx && spitch == nx)
        return cudaMemcpyAsync(dst, src, (size_t)rows * nx * 4, cudaMemcpyDefault, s);
    return cudaMemcpy2DAsync(dst, (size_t)dpitch * 4, src, (size_t)spitch * 4, (size_t)nx * 4, (size_t)rows,
                             cudaMemcpyDefault, s);
}

static pfm_status create_impl(const pfm_desc* desc, const pfm_params* params, void* stream, bool dense,
                              pfm_problem** out);
static pfm_status ensure_copy_stream(pfm_problem* pb);

pfm_status pfm_create(const pfm_desc* desc, const pfm_params* params, void* stream, pfm_problem** out) {
    return create_impl(desc, params, stream, false, out);
}

static pfm_status create_impl(const pfm_desc* desc, const pfm_params* params, void* stream, bool dense,
                              pfm_problem** out) {
    if (!out) return fail(PFM_EINVAL, "out is NULL");
    *out = nullptr;
    DagInfo dag;
    pfm_status st = check_params(params);
    if (st != PFM_OK) return st;
    st = check_desc(desc, &dag);
    if (st != PFM_OK) return st;

    pfm_problem* pb = new pfm_problem();
    pb->ndim = desc->ndim;
    pb->nx = (int)desc->dims[0];
    pb->ny = (int)desc->dims[1];
    pb->nz = (int)desc->dims[2];
    pb->px = row_pitch(pb->nx, dense);
    pb->n = (long long)pb->px * pb->ny * pb->nz;
    pb->nv = (long long)pb->nx * pb->ny * pb->nz;
    pb->nl = dag.nl;
    pb->nn = dag.nn;
    pb->flat = dag.flat;
    pb->prm = *params;
    pb->stream = (cudaStream_t)stream;
    pb->s_node.assign(pb->nn, 1.0f);
    if (desc->s_node)
        for (int A = 0; A < pb->nn; ++A) pb->s_node[A] = desc->s_node[A];
    pb->W.assign((size_t)pb->nn * pb->nl, 0.f);
    for (int A = 0; A < pb->nn; ++A)
        for (int j = 0; j < pb->nl; ++j) pb->W[(size_t)A * pb->nl + j] = (float)dag.W[(size_t)A * pb->nn + dag.leaf_node[j]];

    auto bail = [&](pfm_status s) {
        free_all(pb);
        delete pb;
        return s;
    };
    const size_t ts = elem_size(params->storage);
    const long long n = pb->n;
    const bool fused = params->schedule != PFM_SCHEDULE_INPLACE;
    const bool need_abuf = !fused && params->grad_source == PFM_GRAD_PAPER_LITERAL;
    cudaError_t e;
    for (int k = 0; k < (fused ? 2 : 1); ++k) {
        if ((e = cudaMalloc(&pb->u[k], (size_t)pb->nl * n * ts)) != cudaSuccess) return bail(cuda_fail(e, "alloc u"));
        if ((e = cudaMalloc(&pb->q[k], (size_t)pb->nn * pb->ndim * n * ts)) != cudaSuccess)
            return bail(cuda_fail(e, "alloc q"));
    }
    if (!fused) {
        pb->u[1] = pb->u[0];
        pb->q[1] = pb->q[0];
    }
    if ((e = cudaMalloc(&pb->D, (size_t)pb->nl * n * 4)) != cudaSuccess) return bail(cuda_fail(e, "alloc D"));
    if (desc->S_field && (e = cudaMalloc(&pb->S, (size_t)n * 4)) != cudaSuccess) return bail(cuda_fail(e, "alloc S"));
    if (need_abuf && (e = cudaMalloc(&pb->abuf, (size_t)n * 4)) != cudaSuccess) return bail(cuda_fail(e, "alloc a"));
    pb->energy_blocks = (int)std::min<long long>((n + pfm::ENERGY_NT - 1) / pfm::ENERGY_NT, 152 * 8);
    if ((e = cudaMalloc(&pb->snode_dev, sizeof(float) * pb->nn)) != cudaSuccess) return bail(cuda_fail(e, "alloc"));
    if ((e = cudaMalloc(&pb->flags, sizeof(unsigned))) != cudaSuccess) return bail(cuda_fail(e, "alloc"));
    if ((e = cudaMalloc(&pb->result, sizeof(double) * 2)) != cudaSuccess) return bail(cuda_fail(e, "alloc"));

    cudaStream_t s = pb->stream;
    if ((e = cudaMemsetAsync(pb->flags, 0, sizeof(unsigned), s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
    // the row padding of D and S holds zeros (finite, never read as a voxel)
    if (pb->px != pb->nx) {
        if ((e = cudaMemsetAsync(pb->D, 0, (size_t)pb->nl * n * 4, s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
        if (pb->S && (e = cudaMemsetAsync(pb->S, 0, (size_t)n * 4, s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
    }
    const long long rows = (long long)pb->ny * pb->nz;
    if ((e = copy_rows(pb->D, pb->px, desc->D, pb->nx, pb->nx, pb->nl * rows, s)) != cudaSuccess)
        return bail(cuda_fail(e, "copy D"));
    if (pb->S && (e = copy_rows(pb->S, pb->px, desc->S_field, pb->nx, pb->nx, rows, s)) != cudaSuccess)
        return bail(cuda_fail(e, "copy S"));
    if ((e = cudaMemcpyAsync(pb->snode_dev, pb->s_node.data(), sizeof(float) * pb->nn, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "copy s_node"));
    if ((e = pfm::launch_validate(pb->D, (long long)pb->nl * n, pb->S, n, pb->flags, s)) != cudaSuccess)
        return bail(cuda_fail(e, "validate"));
    pb->launches++;

    const pfm::ProblemView v = view_of(pb);
    const int stor = params->storage;
    if (pb->flat) {
        const int ml = potts_bucket(pb->nl);
        pb->solver = stor == PFM_STORAGE_BF16  ? pfm::make_potts_bf16(ml, pb->ndim, v)
                     : stor == PFM_STORAGE_F16 ? pfm::make_potts_f16(ml, pb->ndim, v)
                                               : pfm::make_potts_f32(ml, pb->ndim, v);
    } else {
        int ml, mn;
        dag_bucket(pb->nl, pb->nn, &ml, &mn);
        pb->solver = stor == PFM_STORAGE_BF16  ? pfm::make_dag_bf16(ml, mn, pb->ndim, v)
                     : stor == PFM_STORAGE_F16 ? pfm::make_dag_f16(ml, mn, pb->ndim, v)
                                               : pfm::make_dag_f32(ml, mn, pb->ndim, v);
    }
    if (!pb->solver) return bail(fail(PFM_EUNSUPPORTED, "no kernel bucket for this problem"));
    // TMA descriptors serve the fused iteration (PFM_SCHEDULE_FUSED only) and
    // the energy reduction (every schedule)
    pb->solver->prepare_tma(pb->u, pb->q, pb->D, pb->S);
    pb->solver->use_tma = params->schedule == PFM_SCHEDULE_FUSED;
    pb->solver->use_tma_inplace = params->schedule == PFM_SCHEDULE_INPLACE;
    pb->zc = model_zc(zc_tiles(pb), pb->nz, device_sms());
    pb->energy_blocks = (int)std::max<long long>(pb->energy_blocks, pb->solver->tma_energy_blocks(pb->zc));
    if ((e = cudaMalloc(&pb->partial, sizeof(double) * 2 * pb->energy_blocks)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc"));
    st = pfm_reset(pb);
    if (st != PFM_OK) return bail(st);
    unsigned f = 0;
    st = read_flags(pb, &f);
    if (st != PFM_OK) return bail(st);
    if (f & pfm::FLAG_BAD_INPUT) return bail(fail(PFM_ENONFINITE, "D not finite or S negative / not finite"));
    *out = pb;
    return PFM_OK;
}

void pfm_destroy(pfm_problem* pb) {
    if (!pb) return;
    cudaStreamSynchronize(pb->stream);
    free_all(pb);
    delete pb;
}

pfm_status pfm_set_data(pfm_problem* pb, const float* D, const float* S_field) {
    if (!pb || !D) return fail(PFM_EINVAL, "NULL argument");
    if ((S_field != nullptr) != (pb->S != nullptr))
        return fail(PFM_EINVAL, "S_field must be given iff the problem was created with one");
    const long long rows = (long long)pb->ny * pb->nz;
    PFM_CUDA(copy_rows(pb->D, pb->px, D, pb->nx, pb->nx, pb->nl * rows, pb->stream), "copy D");
    if (S_field) PFM_CUDA(copy_rows(pb->S, pb->px, S_field, pb->nx, pb->nx, rows, pb->stream), "copy S");
    PFM_CUDA(pfm::launch_validate(pb->D, (long long)pb->nl * pb->n, pb->S, pb->n, pb->flags, pb->stream), "validate");
    pb->launches++;
    return PFM_OK;
}

pfm_status pfm_prefetch_data(pfm_problem* pb, const float* D, const float* S_field) {
    if (!pb || !D) return fail(PFM_EINVAL, "NULL argument");
    if ((S_field != nullptr) != (pb->S != nullptr))
        return fail(PFM_EINVAL, "S_field must be given iff the problem was created with one");
    if (!pb->staged) {
        pfm_status st = ensure_copy_stream(pb);
        if (st != PFM_OK) return st;
        PFM_CUDA(cudaEventCreateWithFlags(&pb->staged, cudaEventDisableTiming), "event");
        PFM_CUDA(cudaEventCreateWithFlags(&pb->consumed, cudaEventDisableTiming), "event");
        PFM_CUDA(cudaEventRecord(pb->consumed, pb->stream), "event");
        // the staging buffers mirror the pitched D and S, padding zeroed once,
        // in copy-stream order ahead of the first copy (a memset on the
        // legacy stream would not be ordered with the non-blocking copy
        // stream, and could land after the copy)
        PFM_CUDA(cudaMalloc(&pb->D_stage, (size_t)pb->nl * pb->n * 4), "alloc staging D");
        PFM_CUDA(cudaMemsetAsync(pb->D_stage, 0, (size_t)pb->nl * pb->n * 4, pb->copy_stream), "memset");
        if (pb->S) {
            PFM_CUDA(cudaMalloc(&pb->S_stage, (size_t)pb->n * 4), "alloc staging S");
            PFM_CUDA(cudaMemsetAsync(pb->S_stage, 0, (size_t)pb->n * 4, pb->copy_stream), "memset");
        }
        PFM_CUDA(cudaMalloc(&pb->stage_flags, sizeof(unsigned)), "alloc staging flags");
    }
    // the staging buffers are free once the work enqueued before the last
    // commit (which may read them: they were D and S then) is done; a
    // prefetch not yet committed is simply overwritten, in copy-stream order
    PFM_CUDA(cudaStreamWaitEvent(pb->copy_stream, pb->consumed, 0), "wait");
    const long long rows = (long long)pb->ny * pb->nz;
    PFM_CUDA(copy_rows(pb->D_stage, pb->px, D, pb->nx, pb->nx, pb->nl * rows, pb->copy_stream), "copy D");
    if (S_field) PFM_CUDA(copy_rows(pb->S_stage, pb->px, S_field, pb->nx, pb->nx, rows, pb->copy_stream), "copy S");
    // validated here, off the compute stream; the commit carries the result over
    PFM_CUDA(cudaMemsetAsync(pb->stage_flags, 0, sizeof(unsigned), pb->copy_stream), "memset");
    PFM_CUDA(pfm::launch_validate(pb->D_stage, (long long)pb->nl * pb->n, pb->S_stage, pb->n, pb->stage_flags,
                                  pb->copy_stream),
             "validate");
    PFM_CUDA(cudaEventRecord(pb->staged, pb->copy_stream), "event");
    pb->stage_pending = true;
    return PFM_OK;
}

pfm_status pfm_commit_data(pfm_problem* pb) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (!pb->stage_pending) return fail(PFM_EINVAL, "no data prefetched since the last commit");
    PFM_CUDA(cudaStreamWaitEvent(pb->stream, pb->staged, 0), "wait");
    if (pb->in_batch) {
        PFM_CUDA(cudaMemcpyAsync(pb->D, pb->D_stage, (size_t)pb->nl * pb->n * 4, cudaMemcpyDeviceToDevice, pb->stream),
                 "move D");
        if (pb->S)
            PFM_CUDA(cudaMemcpyAsync(pb->S, pb->S_stage, (size_t)pb->n * 4, cudaMemcpyDeviceToDevice, pb->stream),
                     "move S");
    } else {
        // the kernels enqueued before this commit still read the old D and S,
        // which become the staging buffers: the next prefetch waits for them
        std::swap(pb->D, pb->D_stage);
        std::swap(pb->S, pb->S_stage);
        pb->solver->set_data(pb->D, pb->S);
        pb->solver->prepare_tma(pb->u, pb->q, pb->D, pb->S);
    }
    PFM_CUDA(pfm::launch_merge_flags(pb->stage_flags, pb->flags, pb->stream), "flags");
    PFM_CUDA(cudaEventRecord(pb->consumed, pb->stream), "event");
    pb->launches++;
    pb->stage_pending = false;
    return PFM_OK;
}

pfm_status pfm_reset(pfm_problem* pb) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    const size_t ts = elem_size(pb->prm.storage);
    pb->cur = 0;
    PFM_CUDA(pfm::launch_init_labels(pb->u[0], pb->prm.storage, pb->nl, pb->n, pb->stream), "init u");
    pb->launches++;
    // both flow buffers: kernels that skip zero-capacity nodes leave their zeros in place
    for (int k = 0; k < (pb->q[1] != pb->q[0] ? 2 : 1); ++k)
        PFM_CUDA(cudaMemsetAsync(pb->q[k], 0, (size_t)pb->nn * pb->ndim * pb->n * ts, pb->stream), "init q");
    pb->iters = 0;
    return PFM_OK;
}

pfm_status pfm_set_step(pfm_problem* pb, double c, double tau) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (!(c > 0) || !isfinite(c) || !(tau > 0) || !isfinite(tau)) return fail(PFM_EINVAL, "c and tau must be > 0");
    pb->prm.c = c;
    pb->prm.tau = tau;
    pb->solver->set_step((float)c, (float)tau);
    return PFM_OK;
}

pfm_status pfm_iterate(pfm_problem* pb, int n_iters) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (n_iters < 0) return fail(PFM_EINVAL, "n_iters must be >= 0");
    const bool fused = pb->prm.schedule != PFM_SCHEDULE_INPLACE;
    for (int it = 0; it < n_iters; ++it) {
        const int src = pb->cur, dst = fused ? 1 - pb->cur : pb->cur;
        int nlaunch = 0;
        cudaError_t e = pb->solver->step(pb->u[src], pb->u[dst], pb->q[src], pb->q[dst], fused, pb->zc, pb->stream,
                                         &nlaunch);
        pb->launches += nlaunch;
        if (e != cudaSuccess) return cuda_fail(e, "iterate");
        pb->cur = dst;
        pb->iters++;
    }
    return PFM_OK;
}

pfm_status pfm_energy(pfm_problem* pb, double* primal, double* dual) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    int nblocks = 0;
    PFM_CUDA(pb->solver->energy(pb->u[pb->cur], pb->q[pb->cur], pb->partial, pb->energy_blocks, pb->zc, pb->stream,
                                &nblocks),
             "energy");
    PFM_CUDA(pfm::launch_energy_final(pb->partial, nblocks, pb->result, pb->flags, pb->stream), "energy");
    pb->launches += 2;
    double h[2];
    PFM_CUDA(cudaMemcpyAsync(h, pb->result, sizeof h, cudaMemcpyDeviceToHost, pb->stream), "read energy");
    unsigned f = 0;
    pfm_status st = read_flags(pb, &f);
    if (st != PFM_OK) return st;
    if (primal) *primal = h[0];
    if (dual) *dual = h[1];
    return flags_status(f);
}

pfm_status pfm_iterate_energy(pfm_problem* pb, int n_iters, double* primal, double* dual) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (n_iters < 1) return fail(PFM_EINVAL, "n_iters must be >= 1");
    pfm_status st = pfm_iterate(pb, n_iters - 1);
    if (st != PFM_OK) return st;
    const bool fused = pb->prm.schedule != PFM_SCHEDULE_INPLACE;
    const int src = pb->cur, dst = fused ? 1 - pb->cur : pb->cur;
    int nlaunch = 0, nblocks = 0;
    if (pb->solver->fuses_energy(fused)) {
        // the last iteration reduces its own input while it streams it
        PFM_CUDA(pb->solver->step(pb->u[src], pb->u[dst], pb->q[src], pb->q[dst], fused, pb->zc, pb->stream,
                                  &nlaunch, pb->partial, &nblocks),
                 "iterate");
        pb->launches += nlaunch;
    } else {
        // separate reduction of the input, queued ahead of the last iteration
        PFM_CUDA(pb->solver->energy(pb->u[src], pb->q[src], pb->partial, pb->energy_blocks, pb->zc, pb->stream,
                                    &nblocks),
                 "energy");
        PFM_CUDA(pb->solver->step(pb->u[src], pb->u[dst], pb->q[src], pb->q[dst], fused, pb->zc, pb->stream,
                                  &nlaunch),
                 "iterate");
        pb->launches += 1 + nlaunch;
    }
    pb->cur = dst;
    pb->iters++;
    PFM_CUDA(pfm::launch_energy_final(pb->partial, nblocks, pb->result, pb->flags, pb->stream), "energy");
    pb->launches++;
    double h[2];
    PFM_CUDA(cudaMemcpyAsync(h, pb->result, sizeof h, cudaMemcpyDeviceToHost, pb->stream), "read energy");
    unsigned f = 0;
    st = read_flags(pb, &f);
    if (st != PFM_OK) return st;
    if (primal) *primal = h[0];
    if (dual) *dual = h[1];
    return flags_status(f);
}

pfm_status pfm_run_to_gap(pfm_problem* pb, int max_iters, int* iters_done, double* rel_gap) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    int done = 0;
    double gap = INFINITY;
    pfm_status st = PFM_OK;
    while (done < max_iters) {
        const int k = std::min(pb->prm.check_every, max_iters - done);
        double E, P;
        st = pfm_iterate_energy(pb, k, &E, &P);
        if (st != PFM_OK) break;
        done += k;
        gap = (E - P) / fabs(E);
        if (gap <= pb->prm.gap_tol) break;
    }
    if (iters_done) *iters_done = done;
    if (rel_gap) *rel_gap = gap;
    if (st != PFM_OK) return st;
    if (!(gap <= pb->prm.gap_tol)) return fail(PFM_ENOTCONVERGED, "gap %.3g above target after %d iterations", gap, done);
    return PFM_OK;
}

pfm_status pfm_get_labels(pfm_problem* pb, float* dst) {
    if (!pb || !dst) return fail(PFM_EINVAL, "NULL argument");
    const long long rows = (long long)pb->nl * pb->ny * pb->nz;
    const long long count = (long long)pb->nl * pb->nv;
    if (pb->prm.storage == PFM_STORAGE_F32) {
        PFM_CUDA(copy_rows(dst, pb->nx, pb->u[pb->cur], pb->px, pb->nx, rows, pb->stream), "copy labels");
    } else {
        float* tmp = nullptr;
        cudaPointerAttributes at{};
        const bool dev = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (dev) {
            tmp = dst;
        } else {
            PFM_CUDA(cudaMallocAsync((void**)&tmp, count * 4, pb->stream), "alloc staging");
        }
        cudaError_t e = pfm::launch_to_f32(pb->u[pb->cur], pb->prm.storage, rows, pb->nx, pb->px, tmp, pb->stream);
        pb->launches++;
        if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(dst, tmp, count * 4, cudaMemcpyDefault, pb->stream);
        if (!dev) cudaFreeAsync(tmp, pb->stream);
        if (e != cudaSuccess) return cuda_fail(e, "labels");
    }
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    return PFM_OK;
}

pfm_status pfm_get_flows(pfm_problem* pb, float* dst) {
    if (!pb || !dst) return fail(PFM_EINVAL, "NULL argument");
    const long long rows = (long long)pb->nn * pb->ndim * pb->ny * pb->nz;
    const long long count = (long long)pb->nn * pb->ndim * pb->nv;
    if (pb->prm.storage == PFM_STORAGE_F32) {
        PFM_CUDA(copy_rows(dst, pb->nx, pb->q[pb->cur], pb->px, pb->nx, rows, pb->stream), "copy flows");
    } else {
        float* tmp = nullptr;
        cudaPointerAttributes at{};
        const bool dev = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (dev) {
            tmp = dst;
        } else {
            PFM_CUDA(cudaMallocAsync((void**)&tmp, count * 4, pb->stream), "alloc staging");
        }
        cudaError_t e = pfm::launch_to_f32(pb->q[pb->cur], pb->prm.storage, rows, pb->nx, pb->px, tmp, pb->stream);
        pb->launches++;
        if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(dst, tmp, count * 4, cudaMemcpyDefault, pb->stream);
        if (!dev) cudaFreeAsync(tmp, pb->stream);
        if (e != cudaSuccess) return cuda_fail(e, "flows");
    }
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    return PFM_OK;
}

pfm_status pfm_get_state_async(pfm_problem* pb, float* u_dst, float* q_dst) {
    if (!pb || (!u_dst && !q_dst)) return fail(PFM_EINVAL, "NULL argument");
    for (const void* p : {(const void*)u_dst, (const void*)q_dst}) {
        if (!p) continue;
        cudaPointerAttributes at{};
        const bool dev = cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (!dev) return fail(PFM_EINVAL, "pfm_get_state_async needs device destinations");
    }
    const long long zy = (long long)pb->ny * pb->nz;
    if (u_dst) {
        const long long rows = (long long)pb->nl * zy;
        if (pb->prm.storage == PFM_STORAGE_F32) {
            PFM_CUDA(copy_rows(u_dst, pb->nx, pb->u[pb->cur], pb->px, pb->nx, rows, pb->stream), "copy labels");
        } else {
            PFM_CUDA(pfm::launch_to_f32(pb->u[pb->cur], pb->prm.storage, rows, pb->nx, pb->px, u_dst, pb->stream),
                     "labels");
            pb->launches++;
        }
    }
    if (q_dst) {
        const long long rows = (long long)pb->nn * pb->ndim * zy;
        if (pb->prm.storage == PFM_STORAGE_F32) {
            PFM_CUDA(copy_rows(q_dst, pb->nx, pb->q[pb->cur], pb->px, pb->nx, rows, pb->stream), "copy flows");
        } else {
            PFM_CUDA(pfm::launch_to_f32(pb->q[pb->cur], pb->prm.storage, rows, pb->nx, pb->px, q_dst, pb->stream),
                     "flows");
            pb->launches++;
        }
    }
    return PFM_OK;
}

static pfm_status ensure_copy_stream(pfm_problem* pb) {
    if (!pb->copy_stream) PFM_CUDA(cudaStreamCreateWithFlags(&pb->copy_stream, cudaStreamNonBlocking), "copy stream");
    return PFM_OK;
}

pfm_status pfm_get_argmax_async(pfm_problem* pb, int32_t* dst) {
    if (!pb || !dst) return fail(PFM_EINVAL, "NULL argument");
    pfm_status st = ensure_copy_stream(pb);
    if (st != PFM_OK) return st;
    if (!pb->am_buf) {
        PFM_CUDA(cudaMalloc(&pb->am_buf, pb->nv * 4), "alloc argmax buffer");
        PFM_CUDA(cudaEventCreateWithFlags(&pb->am_ready, cudaEventDisableTiming), "event");
        PFM_CUDA(cudaEventCreateWithFlags(&pb->am_done, cudaEventDisableTiming), "event");
        PFM_CUDA(cudaEventRecord(pb->am_done, pb->copy_stream), "event");
    }
    // the previous copy out of the buffer must have landed before it is rewritten
    PFM_CUDA(cudaStreamWaitEvent(pb->stream, pb->am_done, 0), "wait");
    PFM_CUDA(pfm::launch_argmax(pb->u[pb->cur], pb->prm.storage, pb->nl, pb->n, pb->nx, pb->px, pb->nv, pb->am_buf,
                                pb->stream),
             "argmax");
    pb->launches++;
    PFM_CUDA(cudaEventRecord(pb->am_ready, pb->stream), "event");
    PFM_CUDA(cudaStreamWaitEvent(pb->copy_stream, pb->am_ready, 0), "wait");
    PFM_CUDA(cudaMemcpyAsync(dst, pb->am_buf, pb->nv * 4, cudaMemcpyDefault, pb->copy_stream), "copy argmax");
    PFM_CUDA(cudaEventRecord(pb->am_done, pb->copy_stream), "event");
    return PFM_OK;
}

pfm_status pfm_readback_wait(pfm_problem* pb) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (pb->am_done) PFM_CUDA(cudaEventSynchronize(pb->am_done), "wait");
    return PFM_OK;
}

pfm_status pfm_get_argmax(pfm_problem* pb, int32_t* dst) {
    if (!pb || !dst) return fail(PFM_EINVAL, "NULL argument");
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    int* tmp = dev ? (int*)dst : nullptr;
    if (!dev) PFM_CUDA(cudaMallocAsync((void**)&tmp, pb->nv * 4, pb->stream), "alloc staging");
    cudaError_t e =
        pfm::launch_argmax(pb->u[pb->cur], pb->prm.storage, pb->nl, pb->n, pb->nx, pb->px, pb->nv, tmp, pb->stream);
    pb->launches++;
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(dst, tmp, pb->nv * 4, cudaMemcpyDefault, pb->stream);
    if (!dev) cudaFreeAsync(tmp, pb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "argmax");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    return PFM_OK;
}

static pfm_status stage_in(pfm_problem* pb, const float* src, long long count, float** dev_out, bool* owned) {
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    *owned = !dev;
    if (dev) {
        *dev_out = (float*)src;
        return PFM_OK;
    }
    PFM_CUDA(cudaMallocAsync((void**)dev_out, count * 4, pb->stream), "alloc staging");
    PFM_CUDA(cudaMemcpyAsync(*dev_out, src, count * 4, cudaMemcpyDefault, pb->stream), "copy in");
    return PFM_OK;
}

pfm_status pfm_set_labels(pfm_problem* pb, const float* src) {
    if (!pb || !src) return fail(PFM_EINVAL, "NULL argument");
    float* tmp;
    bool owned;
    pfm_status st = stage_in(pb, src, (long long)pb->nl * pb->nv, &tmp, &owned);
    if (st != PFM_OK) return st;
    PFM_CUDA(cudaMemsetAsync(pb->flags, 0, sizeof(unsigned), pb->stream), "memset");
    cudaError_t e = pfm::launch_set_labels(tmp, pb->prm.storage, pb->nl, pb->nv, pb->nx, pb->px, pb->n,
                                           pb->u[pb->cur], pb->flags, pb->stream);
    pb->launches++;
    if (owned) cudaFreeAsync(tmp, pb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set labels");
    unsigned f = 0;
    st = read_flags(pb, &f);
    if (st != PFM_OK) return st;
    if (f) {
        cudaMemsetAsync(pb->flags, 0, sizeof(unsigned), pb->stream);
        cudaStreamSynchronize(pb->stream);
    }
    return flags_status(f);
}

pfm_status pfm_set_flows(pfm_problem* pb, const float* src) {
    if (!pb || !src) return fail(PFM_EINVAL, "NULL argument");
    float* tmp;
    bool owned;
    pfm_status st = stage_in(pb, src, (long long)pb->nn * pb->ndim * pb->nv, &tmp, &owned);
    if (st != PFM_OK) return st;
    cudaError_t e = pfm::launch_set_flows(tmp, pb->prm.storage, pb->nn, pb->ndim, pb->nx, pb->ny, pb->nz, pb->px,
                                          pb->snode_dev, pb->S, pb->prm.norm == PFM_NORM_ANISO, pb->q[pb->cur],
                                          pb->stream);
    pb->launches++;
    if (owned) cudaFreeAsync(tmp, pb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set flows");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    return PFM_OK;
}

static size_t state_bytes(const pfm_problem* pb) {
    const size_t es = elem_size(pb->prm.storage);
    return PFM_STATE_HEADER_BYTES + es * ((size_t)pb->nl * pb->nv + (size_t)pb->nn * pb->ndim * pb->nv);
}

// Copy rows of nx values of es bytes between a dense array and a pitched one.
static cudaError_t copy_rows_es(void* dst, int dpitch, const void* src, int spitch, int nx, long long rows, size_t es,
                                cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, (size_t)dpitch * es, src, (size_t)spitch * es, (size_t)nx * es, (size_t)rows,
                             cudaMemcpyDefault, s);
}

pfm_status pfm_get_state(pfm_problem* pb, void* dst, size_t* size) {
    if (!pb || !size) return fail(PFM_EINVAL, "NULL argument");
    const size_t need = state_bytes(pb);
    if (!dst) {
        *size = need;
        return PFM_OK;
    }
    if (*size < need) return fail(PFM_EINVAL, "state blob needs %zu bytes, %zu given", need, *size);
    pfm_state_header h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "PFMSTATE", 8);
    h.version = PFM_VERSION;
    h.storage = pb->prm.storage;
    h.ndim = pb->ndim;
    h.n_leaf = pb->nl;
    h.n_nodes = pb->nn;
    h.dims[0] = pb->nx;
    h.dims[1] = pb->ny;
    h.dims[2] = pb->nz;
    h.iterations = pb->iters;
    h.c = pb->prm.c;
    h.tau = pb->prm.tau;
    const size_t es = elem_size(pb->prm.storage);
    unsigned char* out = static_cast<unsigned char*>(dst);
    const long long zy = (long long)pb->ny * pb->nz;
    PFM_CUDA(cudaMemcpyAsync(out, &h, sizeof h, cudaMemcpyDefault, pb->stream), "write state header");
    unsigned char* uo = out + PFM_STATE_HEADER_BYTES;
    unsigned char* qo = uo + es * (size_t)pb->nl * pb->nv;
    PFM_CUDA(copy_rows_es(uo, pb->nx, pb->u[pb->cur], pb->px, pb->nx, (long long)pb->nl * zy, es, pb->stream),
             "copy labels");
    PFM_CUDA(copy_rows_es(qo, pb->nx, pb->q[pb->cur], pb->px, pb->nx, (long long)pb->nn * pb->ndim * zy, es,
                          pb->stream),
             "copy flows");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    *size = need;
    return PFM_OK;
}

pfm_status pfm_set_state(pfm_problem* pb, const void* src, size_t size) {
    if (!pb || !src) return fail(PFM_EINVAL, "NULL argument");
    const size_t need = state_bytes(pb);
    if (size < need) return fail(PFM_EINVAL, "state blob of %zu bytes, this problem's state needs %zu", size, need);
    pfm_state_header h;
    PFM_CUDA(cudaMemcpyAsync(&h, src, sizeof h, cudaMemcpyDefault, pb->stream), "read state header");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    if (memcmp(h.magic, "PFMSTATE", 8) != 0) return fail(PFM_EINVAL, "not a state blob (magic)");
    if (h.version != PFM_VERSION) return fail(PFM_EINVAL, "state blob version %d, library %d", h.version, PFM_VERSION);
    if (h.storage != pb->prm.storage) return fail(PFM_EINVAL, "state blob storage %d, problem %d", h.storage,
                                                  pb->prm.storage);
    if (h.ndim != pb->ndim || h.n_leaf != pb->nl || h.n_nodes != pb->nn || h.dims[0] != pb->nx ||
        h.dims[1] != pb->ny || h.dims[2] != pb->nz)
        return fail(PFM_EINVAL, "state blob shape differs from the problem's");
    if (h.iterations < 0 || !(h.c > 0) || !isfinite(h.c) || !(h.tau > 0) || !isfinite(h.tau))
        return fail(PFM_EINVAL, "state blob header out of range");
    const size_t es = elem_size(pb->prm.storage);
    const unsigned char* in = static_cast<const unsigned char*>(src);
    const unsigned char* ui = in + PFM_STATE_HEADER_BYTES;
    const unsigned char* qi = ui + es * (size_t)pb->nl * pb->nv;
    const long long zy = (long long)pb->ny * pb->nz;
    // only the nx columns of each row are written: the row padding keeps its zeros
    PFM_CUDA(copy_rows_es(pb->u[pb->cur], pb->px, ui, pb->nx, pb->nx, (long long)pb->nl * zy, es, pb->stream),
             "copy labels");
    PFM_CUDA(copy_rows_es(pb->q[pb->cur], pb->px, qi, pb->nx, pb->nx, (long long)pb->nn * pb->ndim * zy, es,
                          pb->stream),
             "copy flows");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    pb->iters = h.iterations;
    return pfm_set_step(pb, h.c, h.tau);
}

pfm_status pfm_shape(const pfm_problem* pb, int* ndim, int64_t dims[3], int* n_leaf, int* n_nodes) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (ndim) *ndim = pb->ndim;
    if (dims) {
        dims[0] = pb->nx;
        dims[1] = pb->ny;
        dims[2] = pb->nz;
    }
    if (n_leaf) *n_leaf = pb->nl;
    if (n_nodes) *n_nodes = pb->nn;
    return PFM_OK;
}

const char* pfm_kernel_variant(const pfm_problem* pb) {
    if (!pb || !pb->solver) return "";
    return pb->solver->variant(pb->prm.schedule != PFM_SCHEDULE_INPLACE);
}

pfm_status pfm_adjoint_step(pfm_problem* pb, const float* u_k, const float* q_k, const float* u_k1,
                            const float* ubar_k1, const float* qbar_k1, float* ubar_k, float* qbar_k, float* Dbar,
                            float* Sbar, float* work) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (!u_k || !q_k || !u_k1 || !ubar_k1 || !qbar_k1 || !ubar_k || !qbar_k || !Dbar || !work)
        return fail(PFM_EINVAL, "NULL buffer");
    if (!pb->flat) return fail(PFM_EUNSUPPORTED, "the adjoint covers the Potts model (flat label set)");
    if (pb->nl > 16) return fail(PFM_EUNSUPPORTED, "the adjoint supports at most 16 labels");
    if (pb->prm.grad_source != PFM_GRAD_NORMALISED)
        return fail(PFM_EUNSUPPORTED, "the adjoint differentiates the NORMALISED iteration");
    pfm::AdjLaunch L{};
    L.u_k = u_k;
    L.q_k = q_k;
    L.u_k1 = u_k1;
    L.ubar_k1 = ubar_k1;
    L.qbar_k1 = qbar_k1;
    L.ubar_k = ubar_k;
    L.qbar_k = qbar_k;
    L.Dbar = Dbar;
    L.Sbar = pb->S ? Sbar : nullptr;
    L.ybar = work;
    L.dbar = work + (size_t)pb->nl * pb->ndim * pb->nv;
    L.D = pb->D;
    L.S = pb->S;
    L.nx = pb->nx;
    L.px = pb->px;
    L.np = pb->n;
    L.ny = pb->ny;
    L.nz = pb->nz;
    L.nl = pb->nl;
    L.n = pb->nv;
    L.c = (float)pb->prm.c;
    L.ctau = (float)(pb->prm.c * pb->prm.tau);
    L.aniso = pb->prm.norm == PFM_NORM_ANISO;
    for (int j = 0; j < 16; ++j) L.s_node[j] = j < pb->nl ? pb->s_node[j] : 0.f;
    PFM_CUDA(pfm::launch_adjoint(L, pb->ndim, pb->stream), "adjoint");
    pb->launches += 3;
    return PFM_OK;
}

pfm_status pfm_adjoint_steps(pfm_problem* pb, int n_steps, const float* const* u_states,
                             const float* const* q_states, float* ubar, float* qbar, float* Dbar, float* Sbar,
                             float* work) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (n_steps < 1) return fail(PFM_EINVAL, "n_steps must be >= 1");
    if (!u_states || !q_states || !ubar || !qbar || !Dbar || !work) return fail(PFM_EINVAL, "NULL buffer");
    for (int k = 0; k <= n_steps; ++k)
        if (!u_states[k] || (k < n_steps && !q_states[k])) return fail(PFM_EINVAL, "NULL state");
    if (!pb->flat) return fail(PFM_EUNSUPPORTED, "the adjoint covers the Potts model (flat label set)");
    if (pb->nl > 16) return fail(PFM_EUNSUPPORTED, "the adjoint supports at most 16 labels");
    if (pb->prm.grad_source != PFM_GRAD_NORMALISED)
        return fail(PFM_EUNSUPPORTED, "the adjoint differentiates the NORMALISED iteration");
    std::vector<pfm::AdjLaunch> st((size_t)n_steps);
    for (int k = 0; k < n_steps; ++k) {
        pfm::AdjLaunch& L = st[(size_t)k];
        L = pfm::AdjLaunch{};
        L.u_k = u_states[k];
        L.q_k = q_states[k];
        L.u_k1 = u_states[k + 1];
        L.ubar_k1 = ubar;  // the prox adjoint updates ubar in place, step by step
        L.qbar_k1 = qbar;  // read by the last step's projection adjoint only
        L.ubar_k = ubar;
        L.qbar_k = qbar;   // written by the first step's divergence adjoint only
        L.Dbar = Dbar;
        L.Sbar = pb->S ? Sbar : nullptr;
        L.ybar = work;
        L.dbar = work + (size_t)pb->nl * pb->ndim * pb->nv;
        L.D = pb->D;
        L.S = pb->S;
        L.nx = pb->nx;
        L.px = pb->px;
        L.np = pb->n;
        L.ny = pb->ny;
        L.nz = pb->nz;
        L.nl = pb->nl;
        L.n = pb->nv;
        L.c = (float)pb->prm.c;
        L.ctau = (float)(pb->prm.c * pb->prm.tau);
        L.aniso = pb->prm.norm == PFM_NORM_ANISO;
        for (int j = 0; j < 16; ++j) L.s_node[j] = j < pb->nl ? pb->s_node[j] : 0.f;
    }
    PFM_CUDA(pfm::launch_adjoint_chain(st.data(), n_steps, pb->ndim, pb->stream), "adjoint");
    pb->launches += 2 * n_steps + 1;
    return PFM_OK;
}

pfm_status pfm_selftest_timeout(pfm_problem* pb) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    unsigned before = 0;
    pfm_status st = read_flags(pb, &before);
    if (st != PFM_OK) return st;
    PFM_CUDA(pfm::launch_wait_selftest(pb->flags, pb->stream), "self-test");
    pb->launches++;
    unsigned after = 0;
    if ((st = read_flags(pb, &after)) != PFM_OK) return st;
    // the problem's own state is untouched: restore its flags word
    PFM_CUDA(cudaMemcpyAsync(pb->flags, &before, sizeof before, cudaMemcpyHostToDevice, pb->stream), "flags");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
    if (after & pfm::FLAG_TIMEOUT) return fail(PFM_ETIMEOUT, "a bounded device-side wait expired (self-test)");
    return fail(PFM_ECUDA, "self-test: the bounded wait did not report its timeout");
}

int64_t pfm_iterations_done(const pfm_problem* pb) { return pb ? pb->iters : -1; }
int64_t pfm_launch_count(const pfm_problem* pb) { return pb ? pb->launches : -1; }

// ---------------------------------------------------------------------------
// Batches: many independent problems advanced together by one persistent
// kernel per iteration (work list over all members' tiles); iterations are
// replayed from captured CUDA graphs.
// ---------------------------------------------------------------------------
}  // extern "C"

struct pfm_batch {
    std::vector<pfm_problem*> probs;
    std::vector<pfm::BatchMember> members;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pfm::BatchBase* runner = nullptr;
    int zc = 16;
    int grid = 0;
    int sms = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t launches = 0;
    bool tma = false;   // members run a TMA-staged DAG kernel
    bool dag4 = false;  // ... the four-inner-node one
};

namespace {

constexpr int kGraphIters = 20;  // iterations per captured graph (even: parity preserved)

void batch_drop_graphs(pfm_batch* b) {
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) {
            cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
}

void batch_free(pfm_batch* b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    delete b->runner;
    for (pfm_problem* p : b->probs) pfm_destroy(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

pfm_status batch_setup(pfm_batch* b, int zc, int grid) {
    batch_drop_graphs(b);
    PFM_CUDA(b->runner->setup(b->members.data(), (int)b->members.size(), zc), "batch setup");
    b->zc = zc;
    const int resident = b->runner->ctas_per_sm() * b->sms;
    b->grid = grid > 0 ? grid : std::min(resident, b->runner->n_items());
    return PFM_OK;
}

pfm_status batch_launch_direct(pfm_batch* b, int parity, int n) {
    for (int i = 0; i < n; ++i) {
        PFM_CUDA(b->runner->launch((parity + i) & 1, b->grid, b->stream), "batch launch");
        b->launches++;
    }
    return PFM_OK;
}

}  // namespace

extern "C" {

pfm_status pfm_batch_create(int n, const pfm_desc* descs, const pfm_params* params, void* stream, pfm_batch** out) {
    if (!out) return fail(PFM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !descs) return fail(PFM_EINVAL, "need n >= 1 descriptions");
    pfm_status st = check_params(params);
    if (st != PFM_OK) return st;
    if (params->schedule == PFM_SCHEDULE_INPLACE)
        return fail(PFM_EUNSUPPORTED, "batches use the double-buffered (fused) schedule");
    pfm_batch* b = new pfm_batch();
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        // graph capture needs a stream other than the legacy default stream
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "batch stream");
        }
        b->own_stream = true;
    }
    pfm_params p2 = *params;
    p2.schedule = PFM_SCHEDULE_FUSED_PLAIN;
    int ndim = descs[0].ndim, maxl = 0, maxn = 0;
    bool any_dag = false;
    for (int k = 0; k < n; ++k) {
        if (descs[k].ndim != ndim) {
            batch_free(b);
            return fail(PFM_EINVAL, "all members of a batch need the same ndim");
        }
        pfm_problem* pb = nullptr;
        st = pfm_create(&descs[k], &p2, b->stream, &pb);
        if (st != PFM_OK) {
            const std::string msg = "member " + std::to_string(k) + ": " + g_err;
            batch_free(b);
            return fail(st, "%s", msg.c_str());
        }
        pb->in_batch = true;
        b->probs.push_back(pb);
        maxl = std::max(maxl, pb->nl);
        maxn = std::max(maxn, pb->nn);
        any_dag = any_dag || !pb->flat;
    }
    for (pfm_problem* pb : b->probs) {
        pfm::BatchMember m;
        m.view = view_of(pb);
        for (int k = 0; k < 2; ++k) {
            m.u[k] = pb->u[k];
            m.q[k] = pb->q[k];
        }
        b->members.push_back(m);
    }
    const int stor = params->storage;
    // DAG members on the TMA-staged kernel when every member fits it (the
    // default schedule); PFM_SCHEDULE_FUSED_PLAIN keeps the register-staged one
    if (any_dag && params->schedule == PFM_SCHEDULE_FUSED) {
        // the four-inner-node kernel when every member has at most four
        // non-end-label nodes, else the general TMA DAG kernel
        b->runner = stor == PFM_STORAGE_BF16  ? pfm::make_batch_dag4_tma_bf16(b->members.data(), n, ndim)
                    : stor == PFM_STORAGE_F16 ? pfm::make_batch_dag4_tma_f16(b->members.data(), n, ndim)
                                              : pfm::make_batch_dag4_tma_f32(b->members.data(), n, ndim);
        b->dag4 = b->runner != nullptr;
        if (!b->runner)
            b->runner = stor == PFM_STORAGE_BF16  ? pfm::make_batch_dag_tma_bf16(b->members.data(), n, ndim)
                        : stor == PFM_STORAGE_F16 ? pfm::make_batch_dag_tma_f16(b->members.data(), n, ndim)
                                                  : pfm::make_batch_dag_tma_f32(b->members.data(), n, ndim);
        b->tma = b->runner != nullptr;
    }
    if (!b->runner && !any_dag) {
        const int ml = potts_bucket(maxl);
        b->runner = stor == PFM_STORAGE_BF16  ? pfm::make_batch_potts_bf16(ml, ndim)
                    : stor == PFM_STORAGE_F16 ? pfm::make_batch_potts_f16(ml, ndim)
                                              : pfm::make_batch_potts_f32(ml, ndim);
    } else if (!b->runner) {
        int ml, mn;
        dag_bucket(maxl, maxn, &ml, &mn);
        if (ml)
            b->runner = stor == PFM_STORAGE_BF16  ? pfm::make_batch_dag_bf16(ml, mn, ndim)
                        : stor == PFM_STORAGE_F16 ? pfm::make_batch_dag_f16(ml, mn, ndim)
                                                  : pfm::make_batch_dag_f32(ml, mn, ndim);
    }
    if (!b->runner) {
        batch_free(b);
        return fail(PFM_EUNSUPPORTED, "no batched kernel bucket for these members");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    st = batch_setup(b, 16, 0);
    if (st != PFM_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return PFM_OK;
}

void pfm_batch_destroy(pfm_batch* b) {
    if (b) batch_free(b);
}

int pfm_batch_size(const pfm_batch* b) { return b ? (int)b->probs.size() : 0; }

const char* pfm_batch_kernel_variant(const pfm_batch* b) {
    if (!b) return "";
    return b->dag4 ? "batched_tma_dag4" : b->tma ? "batched_tma_dag" : "batched";
}

pfm_status pfm_batch_member(pfm_batch* b, int index, pfm_problem** out) {
    if (!b || !out || index < 0 || index >= (int)b->probs.size()) return fail(PFM_EINVAL, "bad batch member index");
    *out = b->probs[index];
    return PFM_OK;
}

pfm_status pfm_batch_iterate(pfm_batch* b, int n_iters) {
    if (!b) return fail(PFM_EINVAL, "NULL batch");
    if (n_iters < 0) return fail(PFM_EINVAL, "n_iters must be >= 0");
    const int parity = b->probs[0]->cur;
    int left = n_iters;
    if (left >= kGraphIters) {
        if (!b->graph[parity]) {
            cudaGraph_t g = nullptr;
            PFM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < kGraphIters && e == cudaSuccess; ++i) e = b->runner->launch((parity + i) & 1, b->grid, b->stream);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
            // the captured graph is released on every path (instantiated or not)
            if (g) cudaGraphDestroy(g);
            if (e2 != cudaSuccess) return cuda_fail(e2, "graph capture");
            if (e != cudaSuccess) return cuda_fail(e, "graph capture / instantiate");
        }
        while (left >= kGraphIters) {
            PFM_CUDA(cudaGraphLaunch(b->graph[parity], b->stream), "graph launch");
            b->launches += kGraphIters;
            left -= kGraphIters;
        }
    }
    pfm_status st = batch_launch_direct(b, parity, left);
    if (st != PFM_OK) return st;
    for (pfm_problem* pb : b->probs) {
        pb->cur = (parity + n_iters) & 1;
        pb->iters += n_iters;
    }
    return PFM_OK;
}

pfm_status pfm_batch_energy(pfm_batch* b, double* primal, double* dual) {
    if (!b || !primal || !dual) return fail(PFM_EINVAL, "NULL argument");
    pfm_status first = PFM_OK;
    if (b->runner && b->runner->has_energy()) {
        // one launch over every member's tiles, one reduction per member, one
        // synchronisation for the results and every member's flags
        const size_t n = b->probs.size();
        PFM_CUDA(b->runner->energy(b->probs[0]->cur, b->stream), "batch energy");
        b->launches += 2;
        std::vector<double> h(2 * n);
        std::vector<unsigned> f(n, 0u);
        PFM_CUDA(cudaMemcpyAsync(h.data(), b->runner->energy_out(), sizeof(double) * 2 * n, cudaMemcpyDeviceToHost,
                                 b->stream),
                 "read energy");
        for (size_t k = 0; k < n; ++k)
            PFM_CUDA(cudaMemcpyAsync(&f[k], b->probs[k]->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream),
                     "read flags");
        PFM_CUDA(cudaStreamSynchronize(b->stream), "stream sync");
        for (size_t k = 0; k < n; ++k) {
            primal[k] = h[2 * k];
            dual[k] = h[2 * k + 1];
            const pfm_status st = flags_status(f[k]);
            if (st != PFM_OK && first == PFM_OK) first = st;
        }
        return first;
    }
    for (size_t k = 0; k < b->probs.size(); ++k) {
        pfm_status st = pfm_energy(b->probs[k], &primal[k], &dual[k]);
        if (st != PFM_OK && first == PFM_OK) first = st;
    }
    return first;
}

pfm_status pfm_batch_tune(pfm_batch* b, int trial_iters, int* zc_out, int* grid_out) {
    if (!b) return fail(PFM_EINVAL, "NULL batch");
    if (trial_iters < 1) return fail(PFM_EINVAL, "trial_iters must be >= 1");
    cudaEvent_t e0, e1;
    PFM_CUDA(cudaEventCreate(&e0), "event");
    PFM_CUDA(cudaEventCreate(&e1), "event");
    float best = 3.0e38f;
    int best_zc = b->zc, best_grid = b->grid;
    const int zcs[] = {8, 16, 32, 64};
    pfm_status st = PFM_OK;
    for (int zc : zcs) {
        if ((st = batch_setup(b, zc, 0)) != PFM_OK) break;
        const int resident = b->grid;
        const int grids[] = {resident, std::min(2 * resident, b->runner->n_items()), b->runner->n_items()};
        for (int gi = 0; gi < 3; ++gi) {
            if (gi > 0 && grids[gi] == grids[gi - 1]) continue;
            b->grid = grids[gi];
            const int parity = b->probs[0]->cur;
            if ((st = batch_launch_direct(b, parity, 1)) != PFM_OK) break;  // warm-up
            cudaEventRecord(e0, b->stream);
            if ((st = batch_launch_direct(b, parity + 1, trial_iters)) != PFM_OK) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_zc = zc;
                best_grid = grids[gi];
            }
        }
        if (st != PFM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PFM_OK) return st;
    // the trials advanced the members: start again from the initial state
    for (pfm_problem* pb : b->probs) {
        if ((st = pfm_reset(pb)) != PFM_OK) return st;
    }
    if ((st = batch_setup(b, best_zc, best_grid)) != PFM_OK) return st;
    PFM_CUDA(cudaStreamSynchronize(b->stream), "stream sync");
    if (zc_out) *zc_out = b->zc;
    if (grid_out) *grid_out = b->grid;
    return PFM_OK;
}

int64_t pfm_batch_launch_count(const pfm_batch* b) { return b ? b->launches : -1; }

pfm_status pfm_tune(pfm_problem* pb, int trial_iters, int* zc_out) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (trial_iters < 1) return fail(PFM_EINVAL, "trial_iters must be >= 1");
    std::vector<int> cand = {4, 8, 16, 32, 64, 128, model_zc(zc_tiles(pb), pb->nz, device_sms())};
    for (int& z : cand) z = std::max(1, std::min(z, pb->nz));
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t e0, e1;
    PFM_CUDA(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(PFM_ECUDA, "event");
    }
    const int zc0 = pb->zc;
    float best = 3.0e38f;
    int best_zc = zc0;
    pfm_status st = PFM_OK;
    for (int zc : cand) {
        pb->zc = zc;
        if ((st = pfm_iterate(pb, 1)) != PFM_OK) break;  // warm-up
        cudaEventRecord(e0, pb->stream);
        if ((st = pfm_iterate(pb, trial_iters)) != PFM_OK) break;
        cudaEventRecord(e1, pb->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(PFM_ECUDA, "tune: event sync");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_zc = zc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pb->zc = zc0;
    if (st != PFM_OK) return st;
    if ((st = pfm_set_chunk_length(pb, best_zc)) != PFM_OK) return st;
    // the trials advanced the state: start again from the initial one
    if ((st = pfm_reset(pb)) != PFM_OK) return st;
    unsigned f = 0;
    if ((st = read_flags(pb, &f)) != PFM_OK) return st;
    if ((st = flags_status(f)) != PFM_OK) return st;
    if (zc_out) *zc_out = pb->zc;
    return PFM_OK;
}

pfm_status pfm_set_chunk_length(pfm_problem* pb, int zc) {
    if (!pb) return fail(PFM_EINVAL, "NULL problem");
    if (zc < 1) return fail(PFM_EINVAL, "chunk length must be >= 1");
    zc = std::min(zc, pb->nz);
    // the TMA energy reduction writes one partial per CTA of the chunking
    const long long need = pb->solver->tma_energy_blocks(zc);
    if (need > pb->energy_blocks) {
        PFM_CUDA(cudaStreamSynchronize(pb->stream), "stream sync");
        double* part = nullptr;
        PFM_CUDA(cudaMalloc(&part, sizeof(double) * 2 * need), "alloc");
        cudaFree(pb->partial);
        pb->partial = part;
        pb->energy_blocks = (int)need;
    }
    pb->zc = zc;
    return PFM_OK;
}

int pfm_chunk_length(const pfm_problem* pb) { return pb ? pb->zc : -1; }

pfm_status pfm_select_kernel(pfm_problem* pb, const char* family) {
    if (!pb || !family) return fail(PFM_EINVAL, "NULL argument");
    if (pb->prm.schedule == PFM_SCHEDULE_INPLACE)
        return fail(PFM_EUNSUPPORTED, "kernel families are selectable for the fused schedule only");
    if (!pb->solver->select(family))
        return fail(PFM_EUNSUPPORTED, "kernel family '%s' cannot run this problem", family);
    // the chunk-length model depends on the family's tile
    return pfm_set_chunk_length(pb, model_zc(zc_tiles(pb), pb->nz, device_sms()));
}

// ---------------------------------------------------------------------------
// Explicit-flow ("full-flow") augmented-Lagrangian solver (comparison path).
// ---------------------------------------------------------------------------
}  // extern "C"

struct pfm_alm {
    pfm_problem* pb = nullptr;  // u = pb->u[0], q = pb->q[0], D, S, capacities, energy
    float* pL = nullptr;
    float* pS = nullptr;
    float* f = nullptr;
    double gamma = 0.3, step = 0.2;
    int64_t iters = 0;
};

namespace {

pfm::AlmArgs alm_args(const pfm_alm* m) {
    const pfm_problem* pb = m->pb;
    pfm::AlmArgs a{};
    a.u = (float*)pb->u[0];
    a.q = (float*)pb->q[0];
    a.pL = m->pL;
    a.pS = m->pS;
    a.f = m->f;
    a.D = pb->D;
    a.S = pb->S;
    a.nx = pb->nx;
    a.ny = pb->ny;
    a.nz = pb->nz;
    a.nl = pb->nl;
    a.n = pb->n;
    a.gamma = (float)m->gamma;
    a.step = (float)m->step;
    a.aniso = pb->prm.norm == PFM_NORM_ANISO;
    for (int j = 0; j < 16; ++j) a.s_node[j] = j < pb->nl ? pb->s_node[j] : 0.f;
    return a;
}

void alm_free(pfm_alm* m) {
    if (m->pb) cudaStreamSynchronize(m->pb->stream);
    if (m->pL) cudaFree(m->pL);
    if (m->pS) cudaFree(m->pS);
    if (m->f) cudaFree(m->f);
    cudaGetLastError();
    pfm_destroy(m->pb);
    delete m;
}

}  // namespace

extern "C" {

pfm_status pfm_alm_footprint(const pfm_desc* desc, size_t* device_bytes, int64_t* n_grid_buffers) {
    pfm_params p;
    pfm_params_default(&p);
    p.schedule = PFM_SCHEDULE_INPLACE;
    size_t b = 0;
    int64_t nb = 0;
    int nl = 0;
    pfm_status st = footprint_impl(desc, &p, true, &b, &nb, &nl);
    if (st != PFM_OK) return st;
    const long long n = (long long)desc->dims[0] * desc->dims[1] * desc->dims[2];
    // + sink flows p_L, source flow p_S and the work field f
    if (device_bytes) *device_bytes = b + (size_t)(2 * nl + 1) * n * 4;
    if (n_grid_buffers) *n_grid_buffers = nb + 2 * nl + 1;
    return PFM_OK;
}

pfm_status pfm_alm_create(const pfm_desc* desc, double gamma, double step, int norm, void* stream, pfm_alm** out) {
    if (!out) return fail(PFM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!(gamma > 0) || !(step > 0) || !isfinite(gamma) || !isfinite(step))
        return fail(PFM_EINVAL, "gamma and step must be finite and > 0");
    pfm_params p;
    pfm_params_default(&p);
    p.schedule = PFM_SCHEDULE_INPLACE;
    p.norm = norm;
    pfm_alm* m = new pfm_alm();
    m->gamma = gamma;
    m->step = step;
    pfm_status st = create_impl(desc, &p, stream, true, &m->pb);
    if (st != PFM_OK) {
        delete m;
        return st;
    }
    if (!m->pb->flat || m->pb->nl > 16) {
        alm_free(m);
        return fail(PFM_EUNSUPPORTED, "the explicit-flow solver covers Potts problems with at most 16 labels");
    }
    const size_t n = (size_t)m->pb->n, nl = (size_t)m->pb->nl;
    cudaError_t e;
    if ((e = cudaMalloc(&m->pL, nl * n * 4)) != cudaSuccess || (e = cudaMalloc(&m->pS, n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->f, nl * n * 4)) != cudaSuccess) {
        alm_free(m);
        return cuda_fail(e, "alloc");
    }
    e = pfm::launch_alm_init(alm_args(m), m->pb->stream);
    if (e != cudaSuccess) {
        alm_free(m);
        return cuda_fail(e, "alm init");
    }
    m->pb->launches++;
    *out = m;
    return PFM_OK;
}

void pfm_alm_destroy(pfm_alm* m) {
    if (m) alm_free(m);
}

pfm_status pfm_alm_iterate(pfm_alm* m, int n_iters) {
    if (!m) return fail(PFM_EINVAL, "NULL solver");
    if (n_iters < 0) return fail(PFM_EINVAL, "n_iters must be >= 0");
    const pfm::AlmArgs a = alm_args(m);
    for (int k = 0; k < n_iters; ++k) {
        PFM_CUDA(pfm::launch_alm_iteration(a, m->pb->ndim, m->pb->stream), "alm iterate");
        m->pb->launches += 3;
    }
    m->iters += n_iters;
    return PFM_OK;
}

pfm_status pfm_alm_energy(pfm_alm* m, double* primal, double* dual, double* flow) {
    if (!m) return fail(PFM_EINVAL, "NULL solver");
    pfm_problem* pb = m->pb;
    double E = 0.0, P = 0.0;
    pfm_status st = pfm_energy(pb, &E, &P);
    if (st != PFM_OK && st != PFM_ENONFINITE) return st;
    const int blocks = (int)std::min<long long>((pb->n + 255) / 256, pb->energy_blocks);
    PFM_CUDA(pfm::launch_sum(m->pS, pb->n, pb->partial, blocks, pb->stream), "sum");
    PFM_CUDA(pfm::launch_energy_final(pb->partial, blocks, pb->result, pb->flags, pb->stream), "sum");
    pb->launches += 2;
    double h[2];
    PFM_CUDA(cudaMemcpyAsync(h, pb->result, sizeof h, cudaMemcpyDeviceToHost, pb->stream), "read");
    PFM_CUDA(cudaStreamSynchronize(pb->stream), "sync");
    if (primal) *primal = E;
    if (dual) *dual = P;
    if (flow) *flow = h[0];
    return st;
}

pfm_status pfm_alm_get_labels(pfm_alm* m, float* dst) {
    if (!m) return fail(PFM_EINVAL, "NULL solver");
    return pfm_get_labels(m->pb, dst);
}

int64_t pfm_alm_iterations_done(const pfm_alm* m) { return m ? m->iters : -1; }

}  // extern "C"
