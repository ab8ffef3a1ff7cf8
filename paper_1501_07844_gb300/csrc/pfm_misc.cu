// pfm_misc.cu -- auxiliary kernels: initialisation, readback, checkpoint
// import, input validation and the final FP64 energy reduction.
#include <math.h>

#include "pfm_solver.cuh"

namespace pfm {

namespace {

constexpr int NT = 256;

inline unsigned blocks_for(long long count) { return (unsigned)((count + NT - 1) / NT); }

// Slot of dense element e (rows of nx values) in an array of rows of pitch px
// (32-bit division whenever e fits; the identity without padding).
__device__ __forceinline__ long long slot(long long e, int nx, int px) {
    if (px == nx) return e;
    if (e <= 0xFFFFFFFFll) {
        const unsigned u = (unsigned)e, r = u / (unsigned)nx;
        return (long long)r * px + (u - r * (unsigned)nx);
    }
    const long long r = e / nx;
    return r * px + (e - r * nx);
}

// u_L = 1/#leaves (Algorithm 1 and Algorithm 2, first line).
template <typename T>
__global__ void init_labels_kernel(T* u, int nl, long long n) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= (long long)nl * n) return;
    stu<T>(u + i, 1.0f / nl);
}

// Thresholding of the relaxed labelling: index of the largest u_L, ties to
// the lowest index; out is dense (nv voxels).
template <typename T>
__global__ void argmax_kernel(const T* u, int nl, long long n, int nx, int px, long long nv, int* out) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= nv) return;
    const long long pi = slot(i, nx, px);
    float best = ldv<T>(u + pi);
    int arg = 0;
    for (int j = 1; j < nl; ++j) {
        const float v = ldv<T>(u + (long long)j * n + pi);
        if (v > best) {
            best = v;
            arg = j;
        }
    }
    out[i] = arg;
}

// Pitched rows -> dense FP32 rows (count = rows * nx).
template <typename T>
__global__ void to_f32_kernel(const T* src, long long count, int nx, int px, float* dst) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i < count) dst[i] = ldv<T>(src + slot(i, nx, px));
}

// Checkpoint import of a labelling: entries must be finite and >= 0 with a
// positive sum per voxel; stored as given (the label update is invariant to
// a per-voxel scale, so a labelling read back resumes bit for bit).
template <typename T>
__global__ void set_labels_kernel(const float* src, int nl, long long nv, int nx, int px, long long n, T* dst,
                                  unsigned* flags) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= nv) return;
    float s = 0.f;
    bool ok = true;
    for (int j = 0; j < nl; ++j) {
        const float v = src[(long long)j * nv + i];
        ok = ok && (v >= 0.f) && isfinite(v);
        s += v;
    }
    ok = ok && s > 0.f && isfinite(s);
    if (!ok) {
        atomicOr(flags, FLAG_BAD_LABELS);
        return;
    }
    const long long pi = slot(i, nx, px);
    for (int j = 0; j < nl; ++j) stu<T>(dst + (long long)j * n + pi, src[(long long)j * nv + i]);
}

// Checkpoint import of flows: zero normal flux at the last index of each
// axis, then projection onto the capacity set.
template <typename T, int DIM>
__global__ void set_flows_kernel(const float* src, int nn, int nx, int ny, int nz, int px,
                                 const float* s_node, const float* S, int aniso, T* dst) {
    const long long n = (long long)nx * ny * nz;       // dense voxels of src
    const long long np = (long long)px * ny * nz;      // slots of the pitched S and dst
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;  // voxel
    const int A = blockIdx.y;                                       // node
    if (i >= n) return;
    int x, y, z;
    split3(i, nx, ny, x, y, z);
    const long long pi = ((long long)z * ny + y) * px + x;
    float yv[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) yv[k] = src[((long long)A * DIM + k) * n + i];
    if (x == nx - 1) yv[0] = 0.f;
    if (y == ny - 1) yv[1] = 0.f;
    if constexpr (DIM == 3) {
        if (z == nz - 1) yv[2] = 0.f;
    }
    const float s = s_node[A] * (S ? S[pi] : 1.0f);
    if (aniso) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) yv[k] = fminf(fmaxf(yv[k], -s), s);
    } else {
        // a flow that is feasible up to the rounding of the storage type (e.g.
        // read back from a solver) is kept bit for bit; anything outside is
        // scaled onto the ball
        const float slack = sizeof(T) == 4 ? 1.000001f : 1.02f;  // 16-bit storage: a few ulps
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) r2 = fmaf(yv[k], yv[k], r2);
        if (r2 > s * s * slack || s <= 0.f) {
            const float f = s > 0.f ? s * rsqrtf(r2) : 0.f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) yv[k] *= f;
        }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) stv<T>(dst + ((long long)A * DIM + k) * np + pi, yv[k]);
}

// Self-test of the bounded wait every TMA pipeline uses: an mbarrier that
// nothing arrives on; each thread's wait must give up after its cycle budget
// and raise FLAG_TIMEOUT, and the kernel must return normally.
__global__ void wait_selftest_kernel(unsigned* flags) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the pipelines' wait with a twentieth of their budget (about 0.1 s):
    // the same give-up path, without holding the GPU for the full budget
    const bool ok = mbar_wait_bounded(b, 0u, TMA_WAIT_CYCLES / 20);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
}

__global__ void validate_kernel(const float* D, long long nD, const float* S, long long nS, unsigned* flags) {
    bool bad = false;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < nD; i += (long long)gridDim.x * NT)
        bad = bad || !isfinite(D[i]);
    if (S)
        for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < nS; i += (long long)gridDim.x * NT)
            bad = bad || !(S[i] >= 0.f) || !isfinite(S[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, FLAG_BAD_INPUT);
}

// Sums the per-block (E, P) partials in a fixed order (deterministic).
__global__ void energy_final_kernel(const double* partial, int blocks, double* out, unsigned* flags) {
    __shared__ double sE[1024], sP[1024];
    double E = 0.0, P = 0.0;
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
        E += partial[2 * b];
        P += partial[2 * b + 1];
    }
    sE[threadIdx.x] = E;
    sP[threadIdx.x] = P;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sE[threadIdx.x] += sE[threadIdx.x + w];
            sP[threadIdx.x] += sP[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sE[0];
        out[1] = sP[0];
        if (!isfinite(sE[0]) || !isfinite(sP[0])) atomicOr(flags, FLAG_NONFINITE);
    }
}

}  // namespace

// Runs f(Tag<T>{}) with T the storage type of u and q (0 FP32, 1 BF16, 2 F16).
template <typename T> struct Tag { using type = T; };
template <typename F> void by_storage(int storage, F&& f) {
    if (storage == 0)
        f(Tag<float>{});
    else if (storage == 1)
        f(Tag<__nv_bfloat16>{});
    else
        f(Tag<__half>{});
}

cudaError_t launch_init_labels(void* u, int storage, int nl, long long n, cudaStream_t s) {
    const unsigned b = blocks_for((long long)nl * n);
    by_storage(storage, [&](auto tag) {
        using T = typename decltype(tag)::type;
        init_labels_kernel<T><<<b, NT, 0, s>>>((T*)u, nl, n);
    });
    return cudaGetLastError();
}

cudaError_t launch_argmax(const void* u, int storage, int nl, long long n, int nx, int px, long long nv, int* out,
                          cudaStream_t s) {
    const unsigned b = blocks_for(nv);
    by_storage(storage, [&](auto tag) {
        using T = typename decltype(tag)::type;
        argmax_kernel<T><<<b, NT, 0, s>>>((const T*)u, nl, n, nx, px, nv, out);
    });
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const void* src, int storage, long long rows, int nx, int px, float* dst, cudaStream_t s) {
    const long long count = rows * nx;
    const unsigned b = blocks_for(count);
    by_storage(storage, [&](auto tag) {
        using T = typename decltype(tag)::type;
        to_f32_kernel<T><<<b, NT, 0, s>>>((const T*)src, count, nx, px, dst);
    });
    return cudaGetLastError();
}

cudaError_t launch_set_labels(const float* src, int storage, int nl, long long nv, int nx, int px, long long n,
                              void* dst, unsigned* flags, cudaStream_t s) {
    const unsigned b = blocks_for(nv);
    by_storage(storage, [&](auto tag) {
        using T = typename decltype(tag)::type;
        set_labels_kernel<T><<<b, NT, 0, s>>>(src, nl, nv, nx, px, n, (T*)dst, flags);
    });
    return cudaGetLastError();
}

cudaError_t launch_set_flows(const float* src, int storage, int nn, int ndim, int nx, int ny, int nz, int px,
                             const float* s_node_dev, const float* S, int aniso, void* dst, cudaStream_t s) {
    const dim3 b(blocks_for((long long)nx * ny * nz), (unsigned)nn);  // voxels x nodes (nn <= 16)
    by_storage(storage, [&](auto tag) {
        using T = typename decltype(tag)::type;
        if (ndim == 3)
            set_flows_kernel<T, 3><<<b, NT, 0, s>>>(src, nn, nx, ny, nz, px, s_node_dev, S, aniso, (T*)dst);
        else
            set_flows_kernel<T, 2><<<b, NT, 0, s>>>(src, nn, nx, ny, nz, px, s_node_dev, S, aniso, (T*)dst);
    });
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned* flags, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(flags);
    return cudaGetLastError();
}

__global__ void merge_flags_kernel(const unsigned* src, unsigned* dst) {
    const unsigned f = *src;
    if (f) atomicOr(dst, f);
}

cudaError_t launch_merge_flags(const unsigned* src, unsigned* dst, cudaStream_t s) {
    merge_flags_kernel<<<1, 1, 0, s>>>(src, dst);
    return cudaGetLastError();
}

cudaError_t launch_validate(const float* D, long long nD, const float* S, long long nS, unsigned* flags,
                            cudaStream_t s) {
    validate_kernel<<<1216, NT, 0, s>>>(D, nD, S, nS, flags);
    return cudaGetLastError();
}

cudaError_t launch_energy_final(const double* partial, int blocks, double* out, unsigned* flags, cudaStream_t s) {
    energy_final_kernel<<<1, 1024, 0, s>>>(partial, blocks, out, flags);
    return cudaGetLastError();
}

}  // namespace pfm
