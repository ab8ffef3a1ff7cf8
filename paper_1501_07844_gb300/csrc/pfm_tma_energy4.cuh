// pfm_tma_energy4.cuh -- TMA-staged primal energy E(u) and dual P(q) of a
// DAG problem with at most four non-end-label nodes (the four-inner-node
// kernel's shape: HMF trees, DAGMF), for the gap check of Algorithm 2.
//
// Per voxel x (a8 of the iteration; Eq. dagmf_original for E, the dual
// energy Eq. dagmf_pseudo for P):
//   E = sum_j D_j u_j + sum_A s_A S(x) |grad u_A|,
//       u_A = sum_j W_(A,j) u_j  (an end-label's own node: u_j itself),
//   P = min_j d_j,  d_j = D_j + e_j + sum_A W_(A,j) e_A,  e = div q,
// with forward differences (zero at the last index) and the divergence of
// the zero-flux boundary.  The generic energy kernel forms u_A and d_j as
// dense products over every (node, end-label) pair, one voxel per thread;
// here the work is laid out like the four-inner-node iteration: four
// threads per voxel, lane h with end-labels j = h, h+4, h+8 and inner node
// h; u_A at x, x+1, y+1 and z+1 by four-lane reduce-scatters of the lanes'
// contributions W_(A,j) u_j, the inner divergences broadcast by shuffles.
// The planes of a tile arrive through the same boxes and tensor maps as the
// iteration's (three-stage ring, plane r and r+1 staged together, one block
// barrier per plane); each CTA leaves one (E, P) partial in FP64, summed in
// a fixed order by energy_final_kernel (per problem; for a batch, one launch
// over every member's tiles and energy_final_ranges_kernel).
#pragma once

#include "pfm_tma_dag4.cuh"

namespace pfm {

constexpr int ENERGY4_NT = 4 * FTX * DTY;  // 512 threads: the owned 32 x 4 voxels

// Reduce-scatter of four per-lane values over the voxel's quad: lane h ends
// with part[0] + ... summed over the quad for inner node h (the iteration's
// pattern: the first shuffle step pairs lanes two apart, the second
// neighbours).
__device__ __forceinline__ float quad_reduce_scatter(const float (&part)[DAG4_INNER], int h) {
    const bool hi2 = (h & 2) != 0, hi1 = (h & 1) != 0;
    const float s0 = hi2 ? part[0] : part[2], s1 = hi2 ? part[1] : part[3];
    const float k0 = hi2 ? part[2] : part[0], k1 = hi2 ? part[3] : part[1];
    const float r0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 2);
    const float r1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 2);
    return (hi1 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, hi1 ? r0 : r1, 1);
}

// One tile (bx, by) of z-chunk bz of one problem: E and P of its owned
// voxels into out[0], out[1].  smem: the aligned dynamic shared memory (the
// stages of the problem's layout, then three barriers).  Every thread of the
// CTA calls it.
template <int DIM, typename T>
__device__ __forceinline__ void energy_dag4_tile(const StepArgs<DMAX, DMAX>& a, const TmaMaps& maps,
                                                 const Dag4Shape& sh, int bx, int by, int bz, unsigned char* smem,
                                                 double* out) {
    constexpr int QOFF = 16 / (int)sizeof(T);
    constexpr int ustride = DAG_UY * TMA_BX;
    constexpr int NS = DAG4_SLOTS;
    constexpr int NI = DAG4_INNER;
    __shared__ int s_abort;
    __shared__ double sE[ENERGY4_NT / 32], sP[ENERGY4_NT / 32];
    // scalars read once (the batched kernel's arguments live in global memory)
    const int nl = a.nl, nn = a.nn;
    const int nx = a.nx, ny = a.ny, nz = a.nz, aniso = a.aniso, zc = a.zc;
    const TreeTmaLayout lay(nl, nn, DIM, (int)sizeof(T));
    const int QBX = lay.qbx;
    const int qstride = DAG_QY * QBX;
    const int t = threadIdx.x;
    const int h = t & 3;
    const int v = t >> 2;
    const int x0 = bx * FTX, y0 = by * DTY;
    const int z0 = bz * zc;
    const int z1 = min(z0 + zc, nz);
    const long long n = a.n;
    const long long plane = (long long)a.px * ny;
    const int has_S = a.S != nullptr;
    const unsigned bytes = (unsigned)(nl * ustride * sizeof(T) + nl * ustride * 4 + DIM * nn * qstride * sizeof(T)) +
                           (has_S ? (unsigned)(FTX * DTY * 4) : 0u);
    const unsigned bar0 = smem_addr(smem + lay.g_off);  // the stages only: the barriers follow them
    auto stage_ptr = [&](int k) { return smem + k * lay.stage_bytes; };
    auto issue = [&](int p, int k) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage_ptr(k);
        mbar_expect_tx(bar, bytes);
        tma_load_4d(smem_addr(st + lay.q_off), &maps.q, x0 - QOFF, y0 - 1, p, 0, bar);
        tma_load_4d(smem_addr(st + lay.u_off), &maps.u, x0, y0, p, 0, bar);
        tma_load_4d(smem_addr(st + lay.d_off), &maps.D, x0, y0, p, 0, bar);
        if (has_S) tma_load_3d(smem_addr(st + lay.s_off), &maps.S, x0, y0, p, bar);
    };
    int issued_hi = z0;
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        issue(z0, 0);
        if (z0 + 1 < nz) {
            issue(z0 + 1, 1);
            issued_hi = z0 + 1;
        }
    }
    __syncthreads();

    // the owned voxel of this quad; this lane's end-labels (slot s: j = 4 s + h)
    // and inner node, read once
    const int ex = v & (FTX - 1), ey = v / FTX;
    const int x = x0 + ex, y = y0 + ey;
    const bool own = x < nx && y < ny;
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * QBX + (ex + QOFF);
    const float fx = x < nx - 1 ? 1.f : 0.f, fy = y < ny - 1 ? 1.f : 0.f;
    const int lane0 = (t & 31) & ~3;
    int lnd[NS];
    float capl[NS], wv[NS][NI];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int j = 4 * s + h;
        lnd[s] = j < nl ? sh.lnode[j] : -1;
        capl[s] = j < nl ? a.s_node[lnd[s]] : 0.f;
#pragma unroll
        for (int k = 0; k < NI; ++k) wv[s][k] = j < nl ? sh.w[j][k] : 0.f;
    }
    const int inn = h < sh.ni ? sh.inner[h] : -1;
    const float capi = inn >= 0 ? a.s_node[inn] : 0.f;
    // z flows of plane r-1 (the divergence of plane r closes with them)
    float qzp[NS], qzp_i = 0.f;
#pragma unroll
    for (int s = 0; s < NS; ++s) qzp[s] = 0.f;
    if constexpr (DIM == 3) {
        if (own && z0 > 0) {
            const T* qin = static_cast<const T*>(a.q_in);
            const long long i0 = (long long)(z0 - 1) * plane + (long long)y * a.px + x;
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (lnd[s] >= 0) qzp[s] = ldv<T>(qin + ((long long)lnd[s] * DIM + 2) * n + i0);
            if (inn >= 0) qzp_i = ldv<T>(qin + ((long long)inn * DIM + 2) * n + i0);
        }
    }

    SumF sumE, sumP;
    int r_stop = z0;  // first plane whose stage may still be in flight at an abort
    for (int r = z0; r < z1; ++r) {
        const int s_ = r - z0;
        const int cs = s_ % 3, n1 = (s_ + 1) % 3, n2 = (s_ + 2) % 3;
        // stage n2 held plane r-1, last read before the previous barrier
        if (t == 0 && r + 2 <= z1 && r + 2 < nz) {
            issue(r + 2, n2);
            issued_hi = r + 2;
        }
        bool ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s_ / 3) & 1));
        if (ok && r + 1 < nz) ok = mbar_wait_bounded(bar0 + 8 * n1, (unsigned)(((s_ + 1) / 3) & 1));
        if (!ok) {
            atomicOr(a.flags, FLAG_TIMEOUT);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        const unsigned char* cst = stage_ptr(cs);
        const T* uS = reinterpret_cast<const T*>(cst + lay.u_off);
        const T* uN = reinterpret_cast<const T*>(stage_ptr(n1) + lay.u_off);
        const float* dS = reinterpret_cast<const float*>(cst + lay.d_off);
        const T* qS = reinterpret_cast<const T*>(cst + lay.q_off);
        const float fz = r < nz - 1 ? 1.f : 0.f;
        const float sf = (has_S && own) ? reinterpret_cast<const float*>(cst + lay.s_off)[ey * FTX + ex] : 1.0f;
        // end-labels: data term, own-node gradient norms, contributions to
        // the inner nodes' u at x, x+1, y+1, z+1
        float eData = 0.f, tv = 0.f;
        float p0[NI], px1[NI], py1[NI], pz1[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) p0[k] = px1[k] = py1[k] = pz1[k] = 0.f;
        auto norm = [&](float gx, float gy, float gz) {
            if (aniso) return fabsf(gx) + fabsf(gy) + fabsf(gz);
            return sqrt_approx(fmaf(gz, gz, fmaf(gy, gy, gx * gx)));
        };
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (own && lnd[s] >= 0) {
                const T* uj = uS + (4 * s + h) * ustride + ui;
                const float u0 = lds<T>(uj);
                const float ux = fx != 0.f ? lds<T>(uj + 1) : u0;
                const float uy = fy != 0.f ? lds<T>(uj + TMA_BX) : u0;
                float uz = u0;
                if constexpr (DIM == 3)
                    if (fz != 0.f) uz = lds<T>(uN + (4 * s + h) * ustride + ui);
                eData = fmaf(dS[(4 * s + h) * ustride + ui], u0, eData);
                tv = fmaf(capl[s] * sf, norm(ux - u0, uy - u0, uz - u0), tv);
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    p0[k] = fmaf(wv[s][k], u0, p0[k]);
                    px1[k] = fmaf(wv[s][k], ux, px1[k]);
                    py1[k] = fmaf(wv[s][k], uy, py1[k]);
                    pz1[k] = fmaf(wv[s][k], uz, pz1[k]);
                }
            }
        }
        // inner node h: u_A at x and its neighbours, gradient norm
        const float a0 = quad_reduce_scatter(p0, h);
        const float ax = quad_reduce_scatter(px1, h);
        const float ay = quad_reduce_scatter(py1, h);
        const float az = quad_reduce_scatter(pz1, h);
        if (own && inn >= 0) tv = fmaf(capi * sf, norm(ax - a0, ay - a0, az - a0), tv);
        // dual: divergences (the flux through the far boundary is zero), the
        // end-labels' excess and its minimum over the voxel
        auto divergence = [&](int node, float& qzprev) {
            const T* bx = qS + node * (DIM * qstride) + qi;
            const T* by = bx + qstride;
            float dv = fx * lds<T>(bx) - lds<T>(bx - 1);
            dv += fy * lds<T>(by) - lds<T>(by - QBX);
            if constexpr (DIM == 3) {
                const float qz = lds<T>(bx + 2 * qstride);
                dv += fz * qz - qzprev;
                qzprev = qz;
            }
            return dv;
        };
        float ei = 0.f;
        if (own && inn >= 0) ei = divergence(inn, qzp_i);
        float ep[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) ep[k] = __shfl_sync(0xffffffffu, ei, lane0 + k);
        float dmin = 3.0e38f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (own && lnd[s] >= 0) {
                float dj = dS[(4 * s + h) * ustride + ui] + divergence(lnd[s], qzp[s]);
#pragma unroll
                for (int k = 0; k < NI; ++k) dj = fmaf(wv[s][k], ep[k], dj);
                dmin = fminf(dmin, dj);
            }
        }
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, 1));
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, 2));
        if (own) {
            sumE.add(eData + tv);
            if (h == 0) sumP.add(dmin);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        r_stop = r + 1;
        __syncthreads();
    }
    if (s_abort && t == 0) {
        // planes consumed before the abort are complete (their stages may have
        // been refilled): drain from the first plane not yet consumed
        for (int p = r_stop; p <= issued_hi; ++p) {
            const int s = p - z0;
            mbar_wait_bounded(bar0 + 8 * (s % 3), (unsigned)((s / 3) & 1));
        }
    }
    double accE = sumE.value(), accP = sumP.value();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        accE += __shfl_down_sync(0xffffffffu, accE, off);
        accP += __shfl_down_sync(0xffffffffu, accP, off);
    }
    if ((t & 31) == 0) {
        sE[t >> 5] = accE;
        sP[t >> 5] = accP;
    }
    __syncthreads();
    if (t == 0) {
        double E = 0.0, P = 0.0;
        for (int k = 0; k < ENERGY4_NT / 32; ++k) {
            E += sE[k];
            P += sP[k];
        }
        out[0] = E;
        out[1] = P;
    }
}

// One problem: CTA = (x tile, y tile, z chunk), one partial per CTA.
template <int DIM, typename T>
__global__ void __launch_bounds__(ENERGY4_NT, 1)
energy_dag4_tma_kernel(const StepArgs<DMAX, DMAX> a, const __grid_constant__ TmaMaps maps,
                       const __grid_constant__ Dag4Shape sh, double* partial) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    energy_dag4_tile<DIM, T>(a, maps, sh, blockIdx.x, blockIdx.y, blockIdx.z, dag_smem_base(smem_raw),
                             partial + 2 * b);
}

// The members of a batch: CTA k takes work item k (member, x tile, y tile,
// z chunk) of the batch's list (the items of one member are contiguous), one
// partial per item; args, maps and shapes are per member (one parity).
template <int DIM, typename T>
__global__ void __launch_bounds__(ENERGY4_NT, 1)
batched_energy_dag4_tma_kernel(const StepArgs<DMAX, DMAX>* __restrict__ args, const TmaMaps* __restrict__ maps,
                               const Dag4Shape* __restrict__ shapes, const int4* __restrict__ items,
                               double* partial) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int4 w = items[blockIdx.x];
    energy_dag4_tile<DIM, T>(args[w.x], maps[w.x], shapes[w.x], w.y, w.z, w.w, dag_smem_base(smem_raw),
                             partial + 2 * (long long)blockIdx.x);
}

// Per member k of a batch (block k): the fixed-order sum of its items'
// partials [begin[k], begin[k+1]) into out[2 k], out[2 k + 1]; a non-finite
// result raises FLAG_NONFINITE in the member's flags (args: one parity).
constexpr int ENERGY_RANGES_NT = 256;
static __global__ void __launch_bounds__(ENERGY_RANGES_NT)
energy_final_ranges_kernel(const double* __restrict__ partial, const int* __restrict__ begin,
                           const StepArgs<DMAX, DMAX>* __restrict__ args, double* out) {
    __shared__ double sE[ENERGY_RANGES_NT], sP[ENERGY_RANGES_NT];
    const int k = blockIdx.x;
    const int b0 = begin[k], b1 = begin[k + 1];
    double E = 0.0, P = 0.0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += ENERGY_RANGES_NT) {
        E += partial[2 * (long long)b];
        P += partial[2 * (long long)b + 1];
    }
    sE[threadIdx.x] = E;
    sP[threadIdx.x] = P;
    __syncthreads();
    for (int w = ENERGY_RANGES_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sE[threadIdx.x] += sE[threadIdx.x + w];
            sP[threadIdx.x] += sP[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * k] = sE[0];
        out[2 * k + 1] = sP[0];
        if (!isfinite(sE[0]) || !isfinite(sP[0])) atomicOr(args[k].flags, FLAG_NONFINITE);
    }
}

}  // namespace pfm
