// pfm_noalloc.cu -- pfm_potts_energy_noalloc: the Potts energy / dual
// reduction on caller-held buffers, with its per-block partial sums in a
// fixed device array of this file instead of memory from cudaMalloc.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// an outer allocator that has already claimed the budget (a framework's
// caching allocator, a plugin host), and latency-critical loops where an
// allocation, which can synchronise the device, is not acceptable.  This
// entry point serves them; it allocates nothing and frees nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pfm.h"
#include "pfm_solver.cuh"

namespace pfm {
pfm_status set_error(pfm_status st, const char* msg);
}

namespace {

constexpr int kThreads = pfm::ENERGY_NT;             // voxels per block (one per thread)
constexpr long long kMaxBlocks = 65536;              // => at most 16,777,216 voxels
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: 2 doubles (E, P) per block, then
// one word the final reduction ORs its non-finite flag into (never read: the
// call is asynchronous, so a non-finite E or P reaches the caller as NaN or
// Inf in out).  Every GPU that loads the library holds it (1 MiB) until the
// process exits.
static __device__ __align__(256) double g_scratch[2 * kMaxBlocks + 1];

std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per
// device (host code may not use the symbol itself as an address).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

template <int L, int DIM>
cudaError_t launch(const pfm::StepArgs<L, L>& a, int blocks, double* partial, cudaStream_t s) {
    pfm::energy_partial_kernel<L, L, DIM, false, float><<<blocks, kThreads, 0, s>>>(a, partial);
    return cudaGetLastError();
}

template <int L>
cudaError_t fill_and_launch(int ndim, const int64_t dims[3], int nl, const float* u, const float* q,
                            const float* D, const float* S, const float* s_label, int norm, int blocks,
                            double* partial, cudaStream_t s) {
    pfm::StepArgs<L, L> a{};
    a.u_in = u;
    a.q_in = q;
    a.D = D;
    a.S = S;
    a.nx = (int)dims[0];
    a.px = a.nx;  // the caller's arrays are dense
    a.ny = (int)dims[1];
    a.nz = (int)dims[2];
    a.nl = nl;
    a.nn = nl;
    a.n = (long long)dims[0] * dims[1] * dims[2];
    a.aniso = norm == PFM_NORM_ANISO;
    for (int A = 0; A < L; ++A) a.s_node[A] = A < nl ? (s_label ? s_label[A] : 1.0f) : 0.f;
    return ndim == 3 ? launch<L, 3>(a, blocks, partial, s) : launch<L, 2>(a, blocks, partial, s);
}

}  // namespace

extern "C" pfm_status pfm_potts_energy_noalloc(int ndim, const int64_t dims[3], int n_labels, const float* u,
                                               const float* q, const float* D, const float* S_field,
                                               const float* s_label, int norm, double* out, void* stream) {
    // Host-side checks first; these touch no device.
    using pfm::set_error;
    if (ndim != 2 && ndim != 3) return set_error(PFM_EINVAL, "ndim must be 2 or 3");
    if (!dims || !u || !q || !D || !out) return set_error(PFM_EINVAL, "NULL argument");
    for (int k = 0; k < 3; ++k)
        if (dims[k] < 1 || dims[k] > (1 << 30)) return set_error(PFM_EINVAL, "dims out of range");
    if (ndim == 2 && dims[2] != 1) return set_error(PFM_EINVAL, "2-D problems need dims[2] == 1");
    if (n_labels < 1 || n_labels > 16) return set_error(PFM_EUNSUPPORTED, "n_labels must be 1..16");
    if (norm != PFM_NORM_ISO && norm != PFM_NORM_ANISO) return set_error(PFM_EINVAL, "bad norm");
    if (s_label)
        for (int L = 0; L < n_labels; ++L)
            if (!(s_label[L] >= 0.f) || !(s_label[L] < 3.0e38f))
                return set_error(PFM_EINVAL, "s_label must be finite and >= 0");
    const long long n = (long long)dims[0] * dims[1] * dims[2];
    const long long blocks = (n + kThreads - 1) / kThreads;
    if (blocks > kMaxBlocks)
        return set_error(PFM_EINVAL, "grid exceeds PFM_NOALLOC_MAX_VOXELS (16777216 voxels), the size of the "
                                     "fixed scratch of the allocation-free path");

    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return set_error(PFM_ECUDA, "scratch address lookup failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (n_labels <= 4)
        e = fill_and_launch<4>(ndim, dims, n_labels, u, q, D, S_field, s_label, norm, (int)blocks, scratch, s);
    else if (n_labels <= 8)
        e = fill_and_launch<8>(ndim, dims, n_labels, u, q, D, S_field, s_label, norm, (int)blocks, scratch, s);
    else
        e = fill_and_launch<16>(ndim, dims, n_labels, u, q, D, S_field, s_label, norm, (int)blocks, scratch, s);
    if (e != cudaSuccess) return set_error(PFM_ECUDA, cudaGetErrorString(e));
    unsigned* flag = reinterpret_cast<unsigned*>(scratch + 2 * kMaxBlocks);
    e = pfm::launch_energy_final(scratch, (int)blocks, out, flag, s);
    if (e != cudaSuccess) return set_error(PFM_ECUDA, cudaGetErrorString(e));
    return PFM_OK;
}
