// pfm_alm.cu -- explicit-flow ("full-flow") continuous max-flow for the
// Potts model on the GPU: the augmented-Lagrangian method on the primal of
// Section 3.2 (maximise sum p_S s.t. p_L <= D_L, |q_L| <= S_L,
// div q_L - p_S + p_L = 0, multipliers u_L), with every flow stored.  It is
// the formulation the pseudo-flow method replaces and serves as a same-GPU
// comparison of memory and time.
//
// One iteration (block maximisation of the augmented Lagrangian
//   sum p_S + sum_L <u_L, G_L> - (gamma/2) sum_L |G_L|^2,  G_L = div q_L - p_S + p_L,
// then the multiplier step):
//   K1  f_L = u_L - gamma (div q_L - p_S + p_L)
//   K2  q_L <- Proj(q_L - step grad f_L)                 (projected ascent on q_L)
//   K3  p_L <- min(D_L, p_S - div q_L + u_L / gamma)      (new q_L; closed form)
//       p_S <- (sum_L (div q_L + p_L - u_L / gamma) + 1/gamma) / #L
//       u_L <- u_L - gamma (div q_L - p_S + p_L)
// K1 and K3 are per voxel (the divergence reads x - e_i), K2 reads f at x + e_i.
#include <cuda_runtime.h>

#include "pfm_solver.cuh"

namespace pfm {

namespace {

constexpr int NT = 256;

template <int DIM>
__device__ __forceinline__ float div_at(const float* qa, long long n, long long plane, int nx, int ny, int nz, int x,
                                        int y, int z) {
    float dv = (x < nx - 1 ? qa[0] : 0.f) - (x > 0 ? qa[-1] : 0.f);
    dv += (y < ny - 1 ? qa[n] : 0.f) - (y > 0 ? qa[n - nx] : 0.f);
    if constexpr (DIM == 3) dv += (z < nz - 1 ? qa[2 * n] : 0.f) - (z > 0 ? qa[2 * n - plane] : 0.f);
    return dv;
}

template <int MAXL, int DIM>
__global__ void __launch_bounds__(NT) alm_f_kernel(const AlmArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    split3(i, a.nx, a.ny, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    const float ps = a.pS[i];
#pragma unroll
    for (int L = 0; L < MAXL; ++L) {
        if (L < a.nl) {
            const float dv = div_at<DIM>(a.q + (long long)L * DIM * n + i, n, plane, a.nx, a.ny, a.nz, x, y, z);
            a.f[(long long)L * n + i] = a.u[(long long)L * n + i] - a.gamma * (dv - ps + a.pL[(long long)L * n + i]);
        }
    }
}

template <int MAXL, int DIM>
__global__ void __launch_bounds__(NT) alm_q_kernel(const AlmArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    split3(i, a.nx, a.ny, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    const float sf = a.S ? a.S[i] : 1.0f;
#pragma unroll
    for (int L = 0; L < MAXL; ++L) {
        if (L < a.nl) {
            const float* fl = a.f + (long long)L * n + i;
            const float f0 = fl[0];
            float yv[DIM];
            float* qa = a.q + (long long)L * DIM * n + i;
            yv[0] = qa[0] - a.step * (x < a.nx - 1 ? fl[1] - f0 : 0.f);
            yv[1] = qa[n] - a.step * (y < a.ny - 1 ? fl[a.nx] - f0 : 0.f);
            if constexpr (DIM == 3) yv[2] = qa[2 * n] - a.step * (z < a.nz - 1 ? fl[plane] - f0 : 0.f);
            project<DIM>(yv, a.s_node[L] * sf, a.aniso);
#pragma unroll
            for (int k = 0; k < DIM; ++k) qa[k * n] = yv[k];
        }
    }
}

template <int MAXL, int DIM>
__global__ void __launch_bounds__(NT) alm_p_kernel(const AlmArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    split3(i, a.nx, a.ny, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    const float ps = a.pS[i];
    const float ig = 1.0f / a.gamma;
    float dv[MAXL], pl[MAXL], uu[MAXL];
    float sum = 0.f;
#pragma unroll
    for (int L = 0; L < MAXL; ++L) {
        if (L < a.nl) {
            dv[L] = div_at<DIM>(a.q + (long long)L * DIM * n + i, n, plane, a.nx, a.ny, a.nz, x, y, z);
            uu[L] = a.u[(long long)L * n + i];
            pl[L] = fminf(a.D[(long long)L * n + i], ps - dv[L] + uu[L] * ig);
            sum += dv[L] + pl[L] - uu[L] * ig;
        }
    }
    const float psn = (sum + ig) / a.nl;
    a.pS[i] = psn;
#pragma unroll
    for (int L = 0; L < MAXL; ++L) {
        if (L < a.nl) {
            a.pL[(long long)L * n + i] = pl[L];
            a.u[(long long)L * n + i] = uu[L] - a.gamma * (dv[L] - psn + pl[L]);
        }
    }
}

// p_S initialised to the per-voxel minimum of D, p_L = p_S, u = 1/#L, q = 0.
template <int MAXL>
__global__ void __launch_bounds__(NT) alm_init_kernel(const AlmArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    const long long n = a.n;
    float m = 3.0e38f;
    for (int L = 0; L < a.nl; ++L) m = fminf(m, a.D[(long long)L * n + i]);
    a.pS[i] = m;
    for (int L = 0; L < a.nl; ++L) {
        a.pL[(long long)L * n + i] = m;
        a.u[(long long)L * n + i] = 1.0f / a.nl;
    }
}

__global__ void __launch_bounds__(NT) sum_kernel(const float* v, long long n, double* partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) acc += v[i];
    __shared__ double s[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < NT / 32; ++k) t += s[k];
        partial[2 * blockIdx.x] = t;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

template <int MAXL, int DIM>
cudaError_t launch_iter(const AlmArgs& a, cudaStream_t s) {
    const unsigned b = (unsigned)((a.n + NT - 1) / NT);
    alm_f_kernel<MAXL, DIM><<<b, NT, 0, s>>>(a);
    alm_q_kernel<MAXL, DIM><<<b, NT, 0, s>>>(a);
    alm_p_kernel<MAXL, DIM><<<b, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_alm_init(const AlmArgs& a, cudaStream_t s) {
    const unsigned b = (unsigned)((a.n + NT - 1) / NT);
    alm_init_kernel<16><<<b, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_alm_iteration(const AlmArgs& a, int ndim, cudaStream_t s) {
    const int ml = a.nl <= 4 ? 4 : a.nl <= 8 ? 8 : 16;
    if (ndim == 3) {
        if (ml == 4) return launch_iter<4, 3>(a, s);
        if (ml == 8) return launch_iter<8, 3>(a, s);
        return launch_iter<16, 3>(a, s);
    }
    if (ml == 4) return launch_iter<4, 2>(a, s);
    if (ml == 8) return launch_iter<8, 2>(a, s);
    return launch_iter<16, 2>(a, s);
}

cudaError_t launch_sum(const float* v, long long n, double* partial, int blocks, cudaStream_t s) {
    sum_kernel<<<blocks, NT, 0, s>>>(v, n, partial);
    return cudaGetLastError();
}

}  // namespace pfm
