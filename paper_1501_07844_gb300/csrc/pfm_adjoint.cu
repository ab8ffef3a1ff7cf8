// pfm_adjoint.cu -- reverse-mode (adjoint) step of one Potts iteration.
//
// Forward iteration k (NORMALISED gradient source), per voxel and label j:
//   d_j  = D_j + div q_j                       (q = q^k)
//   u'_j = u_j e_j / a,  e_j = exp(-(d_j - m)/c),  a = sum_l u_l e_l   (u = u^k)
//   y_j  = q_j - c tau grad u'_j
//   q'_j = Proj_{|.| <= s_j S}(y_j)
// Given the adjoints (ubar', qbar') of (u^{k+1}, q^{k+1}), three kernels
// produce (ubar, qbar) of (u^k, q^k) and accumulate Dbar and Sbar:
//   K1 (projection):  ybar_j = J_proj^T qbar'_j,  Sbar += sum_j s_j * dProj/ds . qbar'_j
//   K2 (label prox):  ubar'_j += c tau div ybar_j            (adjoint of -c tau grad)
//                     zbar_j = u'_j (ubar'_j - <u', ubar'>)   (softmax Jacobian)
//                     ubar_j = (e_j / a) (ubar'_j - <u', ubar'>),  dbar_j = -zbar_j / c
//                     Dbar_j += dbar_j
//   K3 (divergence):  qbar_j = ybar_j - grad dbar_j           (adjoint of div is -grad)
// Projection Jacobian (ISO): identity inside the ball; outside,
// (s/|y|)(I - yhat yhat^T) with d/ds = yhat.  ANISO: per component, identity
// inside the box, zero outside with d/ds = sign(y).
#include <cuda_runtime.h>

#include "../../include/pfm.h"
#include "pfm_solver.cuh"

namespace pfm {
pfm_status set_error(pfm_status st, const char* msg);

namespace {

constexpr int NT = 256;

using AdjArgs = AdjLaunch;

// Slot of voxel (x, y, z) in the problem's pitched D and S arrays.
__device__ __forceinline__ long long pitched(const AdjArgs& a, int x, int y, int z) {
    return ((long long)z * a.ny + y) * a.px + x;
}

__device__ __forceinline__ void coords(long long i, int nx, int ny, int& x, int& y, int& z) {
    split3(i, nx, ny, x, y, z);
}

// L: compile-time bound on the label count (4, 8 or 16), so the label loops
// unroll and the per-label values live in registers.  In the prox and
// divergence adjoints every load is unconditional and in bounds (a label
// past nl reads label nl-1, a neighbour past the grid's last index reads the
// voxel itself, which makes its forward difference exactly zero), so the
// loads of all labels issue before the first store; only the stores and
// accumulations are guarded.  The projection adjoint keeps one thread per
// voxel and one label's loads at a time: with all of them in flight (one or
// two threads per voxel) it measured slower.
// Projection adjoint of label j at voxel i (K1): y = q - c tau grad u' from
// the step's flows and output labelling, then ybar = J_proj(y)^T qbar' and
// the derivative of q' with respect to the capacity s, dotted with qbar'.
// Shared by the per-step kernel and the chained kernel, so both apply the
// same arithmetic.
template <int DIM>
__device__ __forceinline__ float proj_adjoint_label(const AdjArgs& a, int j, long long i, int x, int y, int z,
                                                    float sf, const float (&qb)[DIM], float (&yb)[DIM]) {
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    const float* u1 = a.u_k1 + (long long)j * n + i;
    const float g0 = *u1;
    float gr[DIM];
    gr[0] = x < a.nx - 1 ? u1[1] - g0 : 0.f;
    gr[1] = y < a.ny - 1 ? u1[a.nx] - g0 : 0.f;
    if constexpr (DIM == 3) gr[2] = z < a.nz - 1 ? u1[plane] - g0 : 0.f;
    float yv[DIM];
    for (int k = 0; k < DIM; ++k) yv[k] = a.q_k[((long long)j * DIM + k) * n + i] - a.ctau * gr[k];
    const float s = a.s_node[j] * sf;
    float ds = 0.f;  // d q' / d s . qbar'
    if (a.aniso) {
        for (int k = 0; k < DIM; ++k) {
            if (yv[k] > s) {
                yb[k] = 0.f;
                ds += qb[k];
            } else if (yv[k] < -s) {
                yb[k] = 0.f;
                ds -= qb[k];
            } else {
                yb[k] = qb[k];
            }
        }
    } else {
        float r2 = 0.f;
        for (int k = 0; k < DIM; ++k) r2 += yv[k] * yv[k];
        if (r2 > s * s && r2 > 0.f) {
            const float ir = rsqrtf(r2);  // 1 / |y|
            float yq = 0.f;
            for (int k = 0; k < DIM; ++k) yq += yv[k] * qb[k];
            yq *= ir;  // yhat . qbar'
            for (int k = 0; k < DIM; ++k) yb[k] = (s * ir) * (qb[k] - (yv[k] * ir) * yq);
            ds = yq;
        } else {
            for (int k = 0; k < DIM; ++k) yb[k] = qb[k];
        }
    }
    return ds;
}

template <int L, int DIM>
__global__ void __launch_bounds__(NT) adj_proj_kernel(const AdjArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    coords(i, a.nx, a.ny, x, y, z);
    const long long n = a.n;
    const float sf = a.S ? a.S[pitched(a, x, y, z)] : 1.0f;
    float sbar = 0.f;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        if (j >= a.nl) break;
        float qb[DIM], yb[DIM];
        for (int k = 0; k < DIM; ++k) qb[k] = a.qbar_k1[((long long)j * DIM + k) * n + i];
        const float ds = proj_adjoint_label<DIM>(a, j, i, x, y, z, sf, qb, yb);
        for (int k = 0; k < DIM; ++k) a.ybar[((long long)j * DIM + k) * n + i] = yb[k];
        sbar += a.s_node[j] * ds;
    }
    if (a.Sbar) a.Sbar[i] += sbar;
}

// The divergence adjoint of step k (K3: qbar_k = ybar_k - grad dbar_k) and
// the projection adjoint of step k-1 (K1, which reads qbar_k at the voxel
// only) in one pass: qbar_k never goes to memory, ybar_{k-1} overwrites
// ybar_k in the work buffer (each thread reads and writes its own voxel;
// the gradient reads only dbar).  b: step k, a: step k-1 (a.u_k1 = b.u_k).
template <int L, int DIM>
__global__ void __launch_bounds__(NT) adj_div_proj_kernel(const AdjArgs b, const AdjArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    coords(i, a.nx, a.ny, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    const long long o[3] = {x < a.nx - 1 ? 1 : 0, y < a.ny - 1 ? (long long)a.nx : 0,
                            z < a.nz - 1 ? plane : 0};
    const float sf = a.S ? a.S[pitched(a, x, y, z)] : 1.0f;
    float sbar = 0.f;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        if (j >= a.nl) break;
        const float* db = b.dbar + (long long)j * n + i;
        const float d0 = db[0];
        float qb[DIM], yb[DIM];
        for (int k = 0; k < DIM; ++k) qb[k] = b.ybar[((long long)j * DIM + k) * n + i] - (db[o[k]] - d0);
        const float ds = proj_adjoint_label<DIM>(a, j, i, x, y, z, sf, qb, yb);
        for (int k = 0; k < DIM; ++k) a.ybar[((long long)j * DIM + k) * n + i] = yb[k];
        sbar += a.s_node[j] * ds;
    }
    if (a.Sbar) a.Sbar[i] += sbar;
}

// Two threads per voxel, each owning every other label (j = h, h+2, ...):
// half the registers per thread and twice the loads in flight per voxel; the
// per-voxel minimum, <u', ubar'> and the normaliser are combined with one lane
// shuffle each.  Every operand, the accumulated Dbar included, is read
// before the first store (ubar_k may alias ubar_k1: each slot is read, then
// written, by its own thread).
template <int L, int DIM>
__global__ void __launch_bounds__(NT) adj_prox_kernel(const AdjArgs a) {
    constexpr int HL = L / 2;
    const long long gt = (long long)blockIdx.x * NT + threadIdx.x;
    const long long i0 = gt >> 1;
    const int h = (int)(gt & 1);
    const bool live = i0 < a.n;  // both lanes of a pair agree; every lane reaches the shuffles
    const long long i = live ? i0 : a.n - 1;
    int x, y, z;
    coords(i, a.nx, a.ny, x, y, z);
    const long long pi = pitched(a, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    // backward neighbours (the voxel itself at index 0) and the zero normal
    // flow at the last index
    const long long mx = x > 0 ? 1 : 0, my = y > 0 ? a.nx : 0, mz = z > 0 ? plane : 0;
    const float fx = x < a.nx - 1 ? 1.f : 0.f, fy = y < a.ny - 1 ? 1.f : 0.f, fz = z < a.nz - 1 ? 1.f : 0.f;
    const float bx = x > 0 ? 1.f : 0.f, by = y > 0 ? 1.f : 0.f, bz = z > 0 ? 1.f : 0.f;
    float d[HL], ub[HL], u1[HL], uk[HL], db0[HL];
    bool valid[HL];
    const float inv_c = 1.0f / a.c;
    float m = 3.0e38f;
    float dot = 0.f;
#pragma unroll
    for (int k = 0; k < HL; ++k) {
        const int j = h + 2 * k;
        valid[k] = live && j < a.nl;
        const int jl = j < a.nl ? j : a.nl - 1;
        // d_j = D_j + div q_j  (forward recomputation)
        const float* qa = a.q_k + (long long)jl * DIM * n + i;
        float dv = fx * qa[0] - bx * qa[-mx];
        dv += fy * qa[n] - by * qa[n - my];
        if constexpr (DIM == 3) dv += fz * qa[2 * n] - bz * qa[2 * n - mz];
        d[k] = a.D[(long long)jl * a.np + pi] + dv;
        // ubar'_j + c tau div ybar_j
        const float* yb = a.ybar + (long long)jl * DIM * n + i;
        float dy = fx * yb[0] - bx * yb[-mx];
        dy += fy * yb[n] - by * yb[n - my];
        if constexpr (DIM == 3) dy += fz * yb[2 * n] - bz * yb[2 * n - mz];
        ub[k] = a.ubar_k1[(long long)jl * n + i] + a.ctau * dy;
        u1[k] = a.u_k1[(long long)jl * n + i];
        uk[k] = a.u_k[(long long)jl * n + i];
        db0[k] = a.Dbar[(long long)jl * n + i];
        if (valid[k]) {
            m = fminf(m, d[k]);
            dot += u1[k] * ub[k];
        }
    }
    m = fminf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    dot += __shfl_xor_sync(0xffffffffu, dot, 1);
    float asum = 0.f;
#pragma unroll
    for (int k = 0; k < HL; ++k) {
        d[k] = __expf((m - d[k]) * inv_c);  // e_j (shifted)
        if (valid[k]) asum += uk[k] * d[k];
    }
    asum += __shfl_xor_sync(0xffffffffu, asum, 1);
    const float inv_a = 1.0f / asum;
#pragma unroll
    for (int k = 0; k < HL; ++k) {
        const int j = h + 2 * k;
        if (!valid[k]) continue;
        const float w = ub[k] - dot;
        a.ubar_k[(long long)j * n + i] = d[k] * inv_a * w;
        const float dbar = -u1[k] * w * inv_c;
        a.dbar[(long long)j * n + i] = dbar;
        a.Dbar[(long long)j * n + i] = db0[k] + dbar;
    }
}

template <int L, int DIM>
__global__ void __launch_bounds__(NT) adj_div_kernel(const AdjArgs a) {
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= a.n) return;
    int x, y, z;
    coords(i, a.nx, a.ny, x, y, z);
    const long long n = a.n, plane = (long long)a.nx * a.ny;
    // dbar and ybar are the work buffer, which qbar_k does not overlap
    const float* __restrict__ dbar = a.dbar;
    const float* __restrict__ ybar = a.ybar;
    float* __restrict__ qbar = a.qbar_k;
    const long long ox = x < a.nx - 1 ? 1 : 0, oy = y < a.ny - 1 ? a.nx : 0, oz = z < a.nz - 1 ? plane : 0;
    // all loads first
    float dl[L][DIM + 1], yl[L][DIM];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int jl = j < a.nl ? j : a.nl - 1;
        const float* db = dbar + (long long)jl * n + i;
        dl[j][0] = db[0];
        dl[j][1] = db[ox];
        dl[j][2] = db[oy];
        if constexpr (DIM == 3) dl[j][3] = db[oz];
#pragma unroll
        for (int k = 0; k < DIM; ++k) yl[j][k] = ybar[((long long)jl * DIM + k) * n + i];
    }
#pragma unroll
    for (int j = 0; j < L; ++j) {
        if (j < a.nl) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) qbar[((long long)j * DIM + k) * n + i] = yl[j][k] - (dl[j][k + 1] - dl[j][0]);
        }
    }
}

// one thread per voxel for the projection and divergence adjoints, two for
// the prox adjoint (measured: the split pays only where a voxel's per-label
// work is heaviest)
template <int L, int DIM>
void launch3(const AdjArgs& a, cudaStream_t s) {
    const unsigned b1 = (unsigned)((a.n + NT - 1) / NT), b2 = (unsigned)((2 * a.n + NT - 1) / NT);
    adj_proj_kernel<L, DIM><<<b1, NT, 0, s>>>(a);
    adj_prox_kernel<L, DIM><<<b2, NT, 0, s>>>(a);
    adj_div_kernel<L, DIM><<<b1, NT, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_adjoint(const AdjArgs& a, int ndim, cudaStream_t s) {
    const int L = a.nl <= 4 ? 4 : a.nl <= 8 ? 8 : 16;
    if (ndim == 3) {
        if (L == 4) launch3<4, 3>(a, s);
        else if (L == 8) launch3<8, 3>(a, s);
        else launch3<16, 3>(a, s);
    } else {
        if (L == 4) launch3<4, 2>(a, s);
        else if (L == 8) launch3<8, 2>(a, s);
        else launch3<16, 2>(a, s);
    }
    return cudaGetLastError();
}

namespace {

template <int L, int DIM>
cudaError_t launch_chain(const AdjArgs* st, int nsteps, cudaStream_t s) {
    const AdjArgs& last = st[nsteps - 1];
    const unsigned b1 = (unsigned)((last.n + NT - 1) / NT), b2 = (unsigned)((2 * last.n + NT - 1) / NT);
    adj_proj_kernel<L, DIM><<<b1, NT, 0, s>>>(last);
    for (int k = nsteps - 1; k >= 0; --k) {
        adj_prox_kernel<L, DIM><<<b2, NT, 0, s>>>(st[k]);
        if (k > 0)
            adj_div_proj_kernel<L, DIM><<<b1, NT, 0, s>>>(st[k], st[k - 1]);
        else
            adj_div_kernel<L, DIM><<<b1, NT, 0, s>>>(st[0]);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_chain(const AdjArgs* steps, int nsteps, int ndim, cudaStream_t s) {
    const int L = steps[0].nl <= 4 ? 4 : steps[0].nl <= 8 ? 8 : 16;
    if (ndim == 3) return L == 4 ? launch_chain<4, 3>(steps, nsteps, s)
                                 : L == 8 ? launch_chain<8, 3>(steps, nsteps, s) : launch_chain<16, 3>(steps, nsteps, s);
    return L == 4 ? launch_chain<4, 2>(steps, nsteps, s)
                  : L == 8 ? launch_chain<8, 2>(steps, nsteps, s) : launch_chain<16, 2>(steps, nsteps, s);
}

}  // namespace pfm
