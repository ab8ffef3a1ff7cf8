// pfm_device.cuh -- device-side building blocks of libpfm (sm_103a).
//
// Layouts are label-major structure-of-arrays, x fastest, as in pfm.h, with
// rows padded to a pitch px >= nx (a multiple of 8 elements, so that every
// row of the FP32 and 16-bit (BF16, F16) arrays starts on a 16-byte
// boundary, as TMA requires):
//   u[leaf][n], D[leaf][n], q[node][comp][n], S[n];  n = px*ny*nz slots,
//   voxel (x, y, z) at (z*ny + y)*px + x; slots x >= nx are padding that no
//   kernel reads as a voxel.
// A warp covers consecutive x, so every per-label load or store of a warp
// is one contiguous 128-byte (FP32) or 64-byte (BF16, F16) segment.
//
// One iteration at voxel x (Algorithm 1 / Algorithm 2):
//   e_A   = div q_A (+ D_A on end-labels)                    (Section 3.3, d_L)
//   d_j   = sum_A W_(A,j) e_A      (Potts: d_j = e_j)        (path-weight form of d_L)
//   u~_j  = u_j exp(-(d_j - m)/c), m = min_j d_j              (Eq. potts_labelupdate)
//   u_j  <- u~_j / sum u~                                     (normalisation a(x))
//   g_j   = u_j  (NORMALISED)  or  u_j exp(-d_j/c) (PAPER_LITERAL, unshifted)
//   q_A  <- Proj_{|q|<=S_A}(q_A - c tau grad(sum_j W_(A,j) g_j))   (Eq. potts_flowupdate)
// The shift m cancels in the normalised labelling, so it is exact for the
// labelling in both modes; PAPER_LITERAL differentiates the unshifted
// product, as printed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pfm {

// Tile of the fused z-marching kernel: each CTA owns FTX x FTY voxels of
// every plane of a z-chunk and recomputes the labelling on a one-voxel
// halo at +x and +y (the gradient's forward neighbours).
// sqrt(x) by the hardware approximation (relative error about 2^-23; a
// subnormal x counts as 0), for the TV norms of the energy E (the TMA energy
// kernels and the iterations that reduce their input).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int FTX = 32;
constexpr int FTY = 8;
constexpr int FEX = FTX + 1;
constexpr int FEY = FTY + 1;
constexpr int FNE = FEX * FEY;                  // 297 halo-extended voxels
constexpr int FUSED_NT = ((FNE + 31) / 32) * 32;  // 320 threads

constexpr int POINT_NT = 256;                   // threads of the per-voxel kernels

// Device error flags (bitmask in a library-owned word).
enum : unsigned {
    FLAG_NONFINITE = 1u,      // normaliser a(x) not finite or not positive
    FLAG_BAD_INPUT = 2u,      // D not finite, or S negative / not finite
    FLAG_BAD_LABELS = 4u,     // set_labels: negative entry or zero sum
};

template <int MAXL, int MAXN>
struct StepArgs {
    const void* u_in;     // T [nl][n]
    void* u_out;          // T [nl][n]
    const void* q_in;     // T [nn][dim][n]
    void* q_out;          // T [nn][dim][n]
    const float* D;       // [nl][n]
    const float* S;       // [n] or nullptr
    float* abuf;          // [n] normaliser of the unshifted product (in-place PAPER_LITERAL)
    unsigned* flags;
    int nx, ny, nz, nl, nn;
    int px;               // row pitch (elements), >= nx
    int literal, aniso, zc;
    long long n;          // slots per label / component: px*ny*nz
    float inv_c, ctau;
    float s_node[MAXN];
    float W[MAXN][MAXL];  // path weights W_(A,j), node A to end-label j (DAG kernels)
};

template <typename T> __device__ __forceinline__ float ldv(const T* p);
template <> __device__ __forceinline__ float ldv<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ldv<__half>(const __half* p) { return __half2float(__ldg(p)); }
// (x, y, z) of slot i of a volume with rows of `row` slots (nx, or the pitch
// px) and ny rows per plane.  32-bit divisions whenever the index fits: the
// 64-bit division is a long instruction sequence, and a per-element kernel
// that splits its index twice spends most of its issue slots there.
__device__ __forceinline__ void split3(long long i, int row, int ny, int& x, int& y, int& z) {
    if (i <= 0xFFFFFFFFll) {
        const unsigned u = (unsigned)i, r = u / (unsigned)row, zz = r / (unsigned)ny;
        x = (int)(u - r * (unsigned)row);
        y = (int)(r - zz * (unsigned)ny);
        z = (int)zz;
    } else {
        const long long r = i / row, zz = r / ny;
        x = (int)(i - r * row);
        y = (int)(r - zz * ny);
        z = (int)zz;
    }
}

template <typename T> __device__ __forceinline__ void stv(T* p, float v);
template <> __device__ __forceinline__ void stv<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void stv<__nv_bfloat16>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}
// F16 storage: values beyond the largest finite F16 (65504) are stored as
// +-65504 (a capacity that large bounds no flow of a labelling in [0, 1]):
// one conversion that rounds to nearest and saturates (a NaN stays NaN).
template <> __device__ __forceinline__ void stv<__half>(__half* p, float v) {
    unsigned short h;
    asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
    *reinterpret_cast<unsigned short*>(p) = h;
}

// Store of a labelling value.  With F16 storage a value below the smallest
// positive F16 subnormal (2^-24) would round to zero, and the multiplicative
// label update never brings a zero back (FP32 and FP64 reach zero only some
// hundred orders of magnitude later): u is stored as max(u, 2^-24) there.
// This floor is a deviation from the method, stated with its results.
constexpr float F16_U_FLOOR = 5.9604644775390625e-08f;
template <typename T> __device__ __forceinline__ void stu(T* p, float v) {
    if constexpr (std::is_same<T, __half>::value) v = fmaxf(v, F16_U_FLOOR);
    stv<T>(p, v);
}

// Projection onto {|y| <= s}: Euclidean ball (ISO) or box (ANISO).  A zero
// capacity maps every y to exactly 0 (|y|^2 of a tiny y may underflow).
template <int DIM>
__device__ __forceinline__ void project(float (&y)[DIM], float s, int aniso) {
    if (aniso) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) y[k] = fminf(fmaxf(y[k], -s), s);
    } else {
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) r2 = fmaf(y[k], y[k], r2);
        if (r2 > s * s || s <= 0.f) {
            const float f = s > 0.f ? s * rsqrtf(r2) : 0.f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) y[k] *= f;
        }
    }
}

// Label prox at one voxel: from the excesses e_A of all nodes and the old
// labelling u_j, produce the new labelling (in u) and the field the flow
// step differentiates (in g).  Returns false if the normaliser is unusable.
// e_A holds div q_A only; the data term enters through the end-label
// itself (W_(L,L) = 1 and an end-label has no other descendant).
template <int MAXL, int MAXN, bool IS_DAG>
__device__ __forceinline__ bool label_prox(const StepArgs<MAXL, MAXN>& a, const float (&e)[MAXN],
                                           const float (&Dv)[MAXL], float (&u)[MAXL], float (&g)[MAXL],
                                           float& norm_out) {
    static_assert(IS_DAG || MAXL == MAXN, "Potts: one node per label");
    float d[MAXL];
#pragma unroll
    for (int j = 0; j < MAXL; ++j) {
        if constexpr (IS_DAG) {
            float s = Dv[j];
#pragma unroll
            for (int A = 0; A < MAXN; ++A)
                if (A < a.nn) s = fmaf(a.W[A][j], e[A], s);
            d[j] = s;
        } else {
            d[j] = e[j] + Dv[j];
        }
    }
    float m = 3.0e38f;
    if (!a.literal) {
#pragma unroll
        for (int j = 0; j < MAXL; ++j)
            if (j < a.nl) m = fminf(m, d[j]);
    } else {
        m = 0.f;
    }
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < MAXL; ++j) {
        if (j < a.nl) {
            u[j] = u[j] * __expf(-(d[j] - m) * a.inv_c);
            sum += u[j];
        }
    }
    const bool ok = (sum > 0.f) && (sum <= 3.0e38f);
    const float inv = 1.0f / sum;
#pragma unroll
    for (int j = 0; j < MAXL; ++j) {
        if (j < a.nl) {
            const float ut = u[j];
            u[j] = ut * inv;
            g[j] = a.literal ? ut : u[j];
        }
    }
    norm_out = sum;
    return ok;
}

// ---------------------------------------------------------------------------
// Fused z-marching iteration (PFM_SCHEDULE_FUSED): reads (u_in, q_in), writes
// (u_out, q_out).  CTA = (x tile, y tile, z chunk).  Per plane p of the
// chunk: label prox of plane p on the halo-extended tile (results to shared
// memory), then the flow step of plane p-1, whose z-gradient needs plane p.
// ---------------------------------------------------------------------------
// One tile (bx, by) of z-chunk bz; sg = [3][MAXL][FNE] shared floats (the
// field g of three planes).  Every thread of the CTA must call it.
template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__device__ __forceinline__ void fused_tile(const StepArgs<MAXL, MAXN>& a, int bx, int by, int bz, float* sg) {
    const int t = threadIdx.x;
    const bool inE = t < FNE;
    const int ex = t % FEX, ey = t / FEX;
    const int x = bx * FTX + ex;
    const int y = by * FTY + ey;
    const bool valid = inE && x < a.nx && y < a.ny;
    const bool owner = valid && ex < FTX && ey < FTY;
    const int z0 = bz * a.zc;
    const int z1 = min(z0 + a.zc, a.nz);
    const long long n = a.n;
    const long long plane = (long long)a.px * a.ny;
    const T* __restrict__ uin = static_cast<const T*>(a.u_in);
    const T* __restrict__ qin = static_cast<const T*>(a.q_in);
    T* __restrict__ uout = static_cast<T*>(a.u_out);
    T* __restrict__ qout = static_cast<T*>(a.q_out);

    float qk[MAXN][DIM];   // flows of plane p-1 at this voxel
    float gprev[MAXL];     // field g of plane p-1 at this voxel
#pragma unroll
    for (int A = 0; A < MAXN; ++A)
#pragma unroll
        for (int k = 0; k < DIM; ++k) qk[A][k] = 0.f;
#pragma unroll
    for (int j = 0; j < MAXL; ++j) gprev[j] = 0.f;
    if constexpr (DIM == 3) {
        if (valid && z0 > 0) {
            const long long i = (long long)(z0 - 1) * plane + (long long)y * a.px + x;
#pragma unroll
            for (int A = 0; A < MAXN; ++A)
                if (A < a.nn) qk[A][2] = ldv<T>(qin + ((long long)A * DIM + 2) * n + i);
        }
    }
    bool bad = false;
    for (int p = z0; p <= z1; ++p) {
        float qn[MAXN][DIM];
        float gcur[MAXL];
#pragma unroll
        for (int j = 0; j < MAXL; ++j) gcur[j] = 0.f;
        if (p < a.nz && valid) {
            const long long i = (long long)p * plane + (long long)y * a.px + x;
            float u[MAXL], e[MAXN], Dv[MAXL];
            float qxm[MAXN], qym[MAXN];
#pragma unroll
            for (int j = 0; j < MAXL; ++j) {
                if (j < a.nl) {
                    u[j] = ldv<T>(uin + (long long)j * n + i);
                    Dv[j] = __ldg(a.D + (long long)j * n + i);
                } else {
                    u[j] = 0.f;
                    Dv[j] = 0.f;
                }
            }
#pragma unroll
            for (int A = 0; A < MAXN; ++A) {
                if (A < a.nn) {
                    const T* qa = qin + (long long)A * DIM * n + i;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) qn[A][k] = ldv<T>(qa + k * n);
                    qxm[A] = x > 0 ? ldv<T>(qa - 1) : 0.f;
                    qym[A] = y > 0 ? ldv<T>(qa + n - a.px) : 0.f;
                } else {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) qn[A][k] = 0.f;
                    qxm[A] = qym[A] = 0.f;
                }
            }
#pragma unroll
            for (int A = 0; A < MAXN; ++A) {
                float dv = (x < a.nx - 1 ? qn[A][0] : 0.f) - qxm[A] + (y < a.ny - 1 ? qn[A][1] : 0.f) - qym[A];
                if constexpr (DIM == 3) dv += (p < a.nz - 1 ? qn[A][2] : 0.f) - (p > 0 ? qk[A][2] : 0.f);
                e[A] = dv;
            }
            float nrm;
            if (!label_prox<MAXL, MAXN, IS_DAG>(a, e, Dv, u, gcur, nrm)) bad = true;
            float* sp = sg + (p % 3) * MAXL * FNE + t;
#pragma unroll
            for (int j = 0; j < MAXL; ++j)
                if (j < a.nl) sp[j * FNE] = gcur[j];
            if (owner && p < z1) {
#pragma unroll
                for (int j = 0; j < MAXL; ++j)
                    if (j < a.nl) stu<T>(uout + (long long)j * n + i, u[j]);
            }
        } else {
#pragma unroll
            for (int A = 0; A < MAXN; ++A)
#pragma unroll
                for (int k = 0; k < DIM; ++k) qn[A][k] = 0.f;
        }
        __syncthreads();
        const int pm = p - 1;
        if (pm >= z0 && owner) {
            const long long i = (long long)pm * plane + (long long)y * a.px + x;
            const float* sp = sg + (pm % 3) * MAXL * FNE + t;
            float gr[MAXL][DIM];
#pragma unroll
            for (int j = 0; j < MAXL; ++j) {
                if (j < a.nl) {
                    gr[j][0] = x < a.nx - 1 ? sp[j * FNE + 1] - gprev[j] : 0.f;
                    gr[j][1] = y < a.ny - 1 ? sp[j * FNE + FEX] - gprev[j] : 0.f;
                    if constexpr (DIM == 3) gr[j][2] = pm < a.nz - 1 ? gcur[j] - gprev[j] : 0.f;
                } else {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) gr[j][k] = 0.f;
                }
            }
            const float sf = a.S ? __ldg(a.S + i) : 1.0f;
#pragma unroll
            for (int A = 0; A < MAXN; ++A) {
                if (A < a.nn) {
                    float yv[DIM];
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        float gA;
                        if constexpr (IS_DAG) {
                            gA = 0.f;
#pragma unroll
                            for (int j = 0; j < MAXL; ++j)
                                if (j < a.nl) gA = fmaf(a.W[A][j], gr[j][k], gA);
                        } else {
                            gA = gr[A][k];
                        }
                        yv[k] = qk[A][k] - a.ctau * gA;
                    }
                    project<DIM>(yv, a.s_node[A] * sf, a.aniso);
                    T* qa = qout + (long long)A * DIM * n + i;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) stv<T>(qa + k * n, yv[k]);
                }
            }
        }
#pragma unroll
        for (int A = 0; A < MAXN; ++A)
#pragma unroll
            for (int k = 0; k < DIM; ++k) qk[A][k] = qn[A][k];
#pragma unroll
        for (int j = 0; j < MAXL; ++j) gprev[j] = gcur[j];
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
}

template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__global__ void __launch_bounds__(FUSED_NT, 1)
fused_step_kernel(const StepArgs<MAXL, MAXN> a) {
    extern __shared__ float sg[];
    fused_tile<MAXL, MAXN, DIM, IS_DAG, T>(a, blockIdx.x, blockIdx.y, blockIdx.z, sg);
}

// ---------------------------------------------------------------------------
// Batched iteration: one persistent launch advances many independent
// volumes (each with its own grid, label DAG and buffers) by one iteration.
// items[k] = (volume, x tile, y tile, z chunk); CTAs take items round-robin
// and stage the volume's arguments in shared memory.  vols[] holds the
// arguments of this launch's parity (inputs / outputs already swapped).
// ---------------------------------------------------------------------------
template <int MAXL, int MAXN>
constexpr size_t batch_smem_bytes() {
    return (sizeof(float) * 3 * MAXL * FNE + 15) / 16 * 16 + sizeof(StepArgs<MAXL, MAXN>);
}

template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__global__ void __launch_bounds__(FUSED_NT, 1)
batched_step_kernel(const StepArgs<MAXL, MAXN>* __restrict__ vols, const int4* __restrict__ items, int n_items) {
    extern __shared__ float sg[];
    using Args = StepArgs<MAXL, MAXN>;
    Args* sa = reinterpret_cast<Args*>(reinterpret_cast<unsigned char*>(sg) +
                                       (sizeof(float) * 3 * MAXL * FNE + 15) / 16 * 16);
    static_assert(sizeof(Args) % 4 == 0, "argument block copied as words");
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        __syncthreads();  // the previous item is done with sa and sg
        const int* src = reinterpret_cast<const int*>(vols + w.x);
        int* dst = reinterpret_cast<int*>(sa);
        for (int k = threadIdx.x; k < (int)(sizeof(Args) / 4); k += blockDim.x) dst[k] = src[k];
        __syncthreads();
        fused_tile<MAXL, MAXN, DIM, IS_DAG, T>(*sa, w.y, w.z, w.w, sg);
    }
}

// ---------------------------------------------------------------------------
// In-place schedule (PFM_SCHEDULE_INPLACE): the label prox rewrites u, then
// the flow step rewrites q.  Each thread reads and writes only its own
// voxel's entries of the array it updates, so in-place is race free.
// ---------------------------------------------------------------------------
template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__global__ void __launch_bounds__(POINT_NT)
prox_inplace_kernel(const StepArgs<MAXL, MAXN> a) {
    const long long n = a.n;
    const long long i = (long long)blockIdx.x * POINT_NT + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    split3(i, a.px, a.ny, x, y, z);
    if (x >= a.nx) return;  // row padding
    const long long plane = (long long)a.px * a.ny;
    T* u = static_cast<T*>(a.u_out);
    const T* q = static_cast<const T*>(a.q_in);
    float uv[MAXL], e[MAXN], g[MAXL], Dv[MAXL];
#pragma unroll
    for (int j = 0; j < MAXL; ++j) {
        uv[j] = j < a.nl ? ldv<T>(u + (long long)j * n + i) : 0.f;
        Dv[j] = j < a.nl ? __ldg(a.D + (long long)j * n + i) : 0.f;
    }
#pragma unroll
    for (int A = 0; A < MAXN; ++A) {
        float dv = 0.f;
        if (A < a.nn) {
            const T* qa = q + (long long)A * DIM * n + i;
            dv = (x < a.nx - 1 ? ldv<T>(qa) : 0.f) - (x > 0 ? ldv<T>(qa - 1) : 0.f);
            dv += (y < a.ny - 1 ? ldv<T>(qa + n) : 0.f) - (y > 0 ? ldv<T>(qa + n - a.px) : 0.f);
            if constexpr (DIM == 3)
                dv += (z < a.nz - 1 ? ldv<T>(qa + 2 * n) : 0.f) - (z > 0 ? ldv<T>(qa + 2 * n - plane) : 0.f);
        }
        e[A] = dv;
    }
    float nrm;
    const bool ok = label_prox<MAXL, MAXN, IS_DAG>(a, e, Dv, uv, g, nrm);
#pragma unroll
    for (int j = 0; j < MAXL; ++j)
        if (j < a.nl) stu<T>(u + (long long)j * n + i, uv[j]);
    if (a.literal) a.abuf[i] = nrm;
    if (!ok) atomicOr(a.flags, FLAG_NONFINITE);
}

template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__global__ void __launch_bounds__(POINT_NT)
flow_inplace_kernel(const StepArgs<MAXL, MAXN> a) {
    const long long n = a.n;
    const long long i = (long long)blockIdx.x * POINT_NT + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    split3(i, a.px, a.ny, x, y, z);
    if (x >= a.nx) return;  // row padding
    const long long plane = (long long)a.px * a.ny;
    const T* u = static_cast<const T*>(a.u_in);
    T* q = static_cast<T*>(a.q_out);
    // g = u (NORMALISED) or u * a(x) (PAPER_LITERAL: the unnormalised product)
    const float a0 = a.literal ? a.abuf[i] : 1.f;
    const float ax = (a.literal && x < a.nx - 1) ? a.abuf[i + 1] : 1.f;
    const float ay = (a.literal && y < a.ny - 1) ? a.abuf[i + a.px] : 1.f;
    float az = 1.f;
    if constexpr (DIM == 3) az = (a.literal && z < a.nz - 1) ? a.abuf[i + plane] : 1.f;
    float gr[MAXL][DIM];
#pragma unroll
    for (int j = 0; j < MAXL; ++j) {
        if (j < a.nl) {
            const T* uj = u + (long long)j * n + i;
            const float g0 = ldv<T>(uj) * a0;
            gr[j][0] = x < a.nx - 1 ? ldv<T>(uj + 1) * ax - g0 : 0.f;
            gr[j][1] = y < a.ny - 1 ? ldv<T>(uj + a.px) * ay - g0 : 0.f;
            if constexpr (DIM == 3) gr[j][2] = z < a.nz - 1 ? ldv<T>(uj + plane) * az - g0 : 0.f;
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k) gr[j][k] = 0.f;
        }
    }
    const float sf = a.S ? __ldg(a.S + i) : 1.0f;
#pragma unroll
    for (int A = 0; A < MAXN; ++A) {
        if (A < a.nn) {
            T* qa = q + (long long)A * DIM * n + i;
            float yv[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                float gA;
                if constexpr (IS_DAG) {
                    gA = 0.f;
#pragma unroll
                    for (int j = 0; j < MAXL; ++j)
                        if (j < a.nl) gA = fmaf(a.W[A][j], gr[j][k], gA);
                } else {
                    gA = gr[A][k];
                }
                yv[k] = ldv<T>(qa + k * n) - a.ctau * gA;
            }
            project<DIM>(yv, a.s_node[A] * sf, a.aniso);
#pragma unroll
            for (int k = 0; k < DIM; ++k) stv<T>(qa + k * n, yv[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// Primal energy and pseudo-flow dual, FP32 per-voxel terms, a compensated
// FP32 partial per thread, FP64 from the warp level up; one (E, P) partial per
// block, summed in fixed order by energy_final_kernel (deterministic for a
// fixed grid).
// ---------------------------------------------------------------------------
constexpr int ENERGY_NT = 256;

// Compensated (Kahan) FP32 running sum for a thread's share of the energy
// reduction (one z-column of voxels): GB300's FP64 pipe is narrow, and a
// double add per voxel and plane costs more than the iteration's own
// arithmetic, so FP64 starts at the warp / block / grid levels of the
// reduction.  The compensation keeps the partial within a few FP32 ulps
// whatever the column length.
struct SumF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};


template <int MAXL, int MAXN, int DIM, bool IS_DAG, typename T>
__global__ void __launch_bounds__(ENERGY_NT, 2)
energy_partial_kernel(const StepArgs<MAXL, MAXN> a, double* partial) {
    const long long n = a.n;
    const long long plane = (long long)a.px * a.ny;
    const T* u = static_cast<const T*>(a.u_in);
    const T* q = static_cast<const T*>(a.q_in);
    SumF sumE, sumP;
    for (long long i = (long long)blockIdx.x * ENERGY_NT + threadIdx.x; i < n;
         i += (long long)gridDim.x * ENERGY_NT) {
        int x, y, z;
        split3(i, a.px, a.ny, x, y, z);
        if (x >= a.nx) continue;  // row padding
        // Every load is unconditional and in bounds (a label or node past the
        // count reads the last one, a neighbour past the grid's last index
        // reads the voxel itself, so its forward difference is exactly 0), so
        // the loads batch; the path weights past the counts are zero.
        const long long ox = x < a.nx - 1 ? 1 : 0, oy = y < a.ny - 1 ? a.px : 0;
        const long long oz = (DIM == 3 && z < a.nz - 1) ? plane : 0;
        const long long mx = x > 0 ? 1 : 0, my = y > 0 ? a.px : 0, mz = (DIM == 3 && z > 0) ? plane : 0;
        const float fx = x < a.nx - 1 ? 1.f : 0.f, fy = y < a.ny - 1 ? 1.f : 0.f, fz = z < a.nz - 1 ? 1.f : 0.f;
        const float bx = x > 0 ? 1.f : 0.f, by = y > 0 ? 1.f : 0.f, bz = z > 0 ? 1.f : 0.f;
        // primal: data term, then the nodes' gradient norms one axis at a
        // time (the end-labels' differences along one axis, 16 values, are
        // live at once instead of all three axes)
        float u0[MAXL];
        float eData = 0.f;
#pragma unroll
        for (int j = 0; j < MAXL; ++j) {
            const int jl = j < a.nl ? j : a.nl - 1;
            u0[j] = ldv<T>(u + (long long)jl * n + i);
            if (j < a.nl) eData = fmaf(__ldg(a.D + (long long)jl * n + i), u0[j], eData);
        }
        const float sf = a.S ? __ldg(a.S + i) : 1.0f;
        float acc[MAXN];  // sum of |g_A,k| (ANISO) or g_A,k^2 (ISO) over the axes so far
#pragma unroll
        for (int A = 0; A < MAXN; ++A) acc[A] = 0.f;
#pragma unroll 1
        for (int k = 0; k < DIM; ++k) {
            const long long off = k == 0 ? ox : k == 1 ? oy : oz;
            float g[MAXL];
#pragma unroll
            for (int j = 0; j < MAXL; ++j) {
                const int jl = j < a.nl ? j : a.nl - 1;
                g[j] = j < a.nl ? ldv<T>(u + (long long)jl * n + i + off) - u0[j] : 0.f;
            }
#pragma unroll
            for (int A = 0; A < MAXN; ++A) {
                float gA;
                if constexpr (IS_DAG) {
                    gA = 0.f;
#pragma unroll
                    for (int j = 0; j < MAXL; ++j) gA = fmaf(a.W[A][j], g[j], gA);
                } else {
                    gA = g[A];
                }
                acc[A] = a.aniso ? acc[A] + fabsf(gA) : (k == 0 ? gA * gA : fmaf(gA, gA, acc[A]));
            }
        }
        float tv = 0.f;
#pragma unroll
        for (int A = 0; A < MAXN; ++A)
            if (A < a.nn) tv = fmaf(a.s_node[A] * sf, a.aniso ? acc[A] : sqrtf(acc[A]), tv);
        // dual: every node's divergence (zero normal flow at the last index),
        // then the end-labels' excess d_j and its minimum
        float e[MAXN];
#pragma unroll
        for (int A = 0; A < MAXN; ++A) {
            const int Al = A < a.nn ? A : a.nn - 1;
            const T* qa = q + (long long)Al * DIM * n + i;
            float dv = fx * ldv<T>(qa) - bx * ldv<T>(qa - mx);
            dv += fy * ldv<T>(qa + n) - by * ldv<T>(qa + n - my);
            if constexpr (DIM == 3) dv += fz * ldv<T>(qa + 2 * n) - bz * ldv<T>(qa + 2 * n - mz);
            e[A] = A < a.nn ? dv : 0.f;
        }
        float dmin = 3.0e38f;
#pragma unroll
        for (int j = 0; j < MAXL; ++j) {
            if (j < a.nl) {
                const float Dj = __ldg(a.D + (long long)j * n + i);
                float dj;
                if constexpr (IS_DAG) {
                    dj = 0.f;
#pragma unroll
                    for (int A = 0; A < MAXN; ++A) dj = fmaf(a.W[A][j], e[A], dj);
                    dj += Dj;  // W_(leaf,leaf) = 1 and D sits on the end-label itself
                } else {
                    dj = e[j] + Dj;
                }
                dmin = fminf(dmin, dj);
            }
        }
        sumE.add(eData + tv);
        sumP.add(dmin);
    }
    // block reduction in fixed order
    double accE = sumE.value(), accP = sumP.value();
    __shared__ double sE[ENERGY_NT / 32], sP[ENERGY_NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        accE += __shfl_down_sync(0xffffffffu, accE, off);
        accP += __shfl_down_sync(0xffffffffu, accP, off);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sE[w] = accE;
        sP[w] = accP;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double E = 0.0, P = 0.0;
        for (int k = 0; k < ENERGY_NT / 32; ++k) {
            E += sE[k];
            P += sP[k];
        }
        partial[2 * blockIdx.x] = E;
        partial[2 * blockIdx.x + 1] = P;
    }
}

}  // namespace pfm
