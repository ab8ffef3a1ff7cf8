// pfm_tma_inplace.cuh -- TMA-staged sweeps of the in-place schedule
// (PFM_SCHEDULE_INPLACE, Potts, NORMALISED): one copy of u and q, as in the
// paper's memory count.  An iteration is two sweeps, each race free because
// a sweep reads neighbours only of the array it does not write, and its
// boxes of the array it writes cover exactly the CTA's own tile:
//   prox sweep: u <- prox(u, D + div q)  (u, D boxes = the tile; q box with
//               the x-1 / y-1 halo; the z-1 flow from a register);
//   flow sweep: q <- Proj(q - c tau grad u)  (u box with the x+1 / y+1
//               halo; q, S boxes = the tile; the z+1 labelling from the
//               next plane's stage).
// Both march a 32 x 8 tile through a z-chunk (three-stage ring, two planes in
// flight, every wait bounded), two threads per voxel (label halves); what a
// voxel needs of the previous plane stays in registers, so a step reads only
// the stage of its own plane.
#pragma once

#include "pfm_tma.cuh"

namespace pfm {

constexpr int INPLACE_TMA_NT = 2 * FTX * FTY;  // 512 threads: two per owned voxel

// Tensor maps of the in-place sweeps (single state buffer).
struct InplaceMaps {
    CUtensorMap u_tile, D_tile, q_halo;  // prox: 32 x 8, 32 x 8, (32 + 2 QOFF) x 10 boxes
    CUtensorMap u_halo, q_tile, S;       // flow: 40 x 9, 32 x 8, 32 x 8 boxes
};

template <int MAXL, int DIM, typename T>
struct InplaceLayout {
    static constexpr int QOFF = 16 / (int)sizeof(T);
    static constexpr int QBX = FTX + 2 * QOFF;
    static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int tile = FTX * FTY;              // 256 voxels
    // prox stage
    static constexpr int p_u = 0;
    static constexpr int p_d = a128(MAXL * tile * (int)sizeof(T));
    static constexpr int p_q = p_d + a128(MAXL * tile * 4);
    static constexpr int p_stage = p_q + a128(DIM * MAXL * TMA_QY * QBX * (int)sizeof(T));
    // flow stage
    static constexpr int f_u = 0;
    static constexpr int f_q = a128(MAXL * TMA_UY * TMA_BX * (int)sizeof(T));
    static constexpr int f_s = f_q + a128(DIM * MAXL * tile * (int)sizeof(T));
    static constexpr int f_stage = f_s + a128(tile * 4);
    static constexpr int p_bar = TMA_STAGES * p_stage;
    static constexpr int f_bar = TMA_STAGES * f_stage;
    static constexpr int p_total = p_bar + 64 + 128;
    static constexpr int f_total = f_bar + 64 + 128;
};

// Label prox sweep.  CTA = (x tile, y tile, z chunk); plane p of the chunk
// lives in stage (p - z0 + 1) % 3, the flows-only plane z0-1 in stage 0.
template <int MAXL, int DIM, typename T, bool EXACT, bool IDX32>
__global__ void __launch_bounds__(INPLACE_TMA_NT, 1)
prox_inplace_tma_kernel(const StepArgs<MAXL, MAXL> a, const __grid_constant__ InplaceMaps maps) {
    constexpr int HL = MAXL / 2;
    using Lay = InplaceLayout<MAXL, DIM, T>;
    constexpr int qstride = TMA_QY * Lay::QBX;
    constexpr int tile = Lay::tile;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x, h = t & 1, v = t >> 1;
    const int nl = EXACT ? MAXL : a.nl;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, a.nz);
    const long long n = a.n, plane = (long long)a.px * a.ny;
    T* __restrict__ u_out = static_cast<T*>(a.u_out);
    const unsigned bar0 = smem_addr(smem + Lay::p_bar);
    const float kexp = -a.inv_c * 1.4426950408889634f;
    const unsigned bytes_q = (unsigned)(DIM * nl * qstride * sizeof(T));
    const unsigned bytes_all = (unsigned)(nl * tile * sizeof(T)) + (unsigned)(nl * tile * 4) + bytes_q;
    auto stage = [&](int k) { return smem + k * Lay::p_stage; };
    auto issue = [&](int p, int k, bool flows_only) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage(k);
        mbar_expect_tx(bar, flows_only ? bytes_q : bytes_all);
        tma_load_4d(smem_addr(st + Lay::p_q), &maps.q_halo, x0 - Lay::QOFF, y0 - 1, p, 0, bar);
        if (!flows_only) {
            tma_load_4d(smem_addr(st + Lay::p_u), &maps.u_tile, x0, y0, p, 0, bar);
            tma_load_4d(smem_addr(st + Lay::p_d), &maps.D_tile, x0, y0, p, 0, bar);
        }
    };
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(z0 - 1, 0, true);
        issue(z0, 1, false);
        if (z0 + 1 < z1) issue(z0 + 1, 2, false);
    }
    __syncthreads();
    const int ex = v & (FTX - 1), ey = v / FTX;
    const int xe = x0 + ex, ye = y0 + ey;
    const bool own = xe < a.nx && ye < a.ny;
    const int qi = (ey + 1) * Lay::QBX + (ex + Lay::QOFF);
    const long long vox = (long long)ye * a.px + xe;
    float qzp[HL];  // z flow of the previous plane at this voxel
#pragma unroll
    for (int i = 0; i < HL; ++i) qzp[i] = 0.f;
    bool ok = mbar_wait_bounded(bar0, 0u);
    if constexpr (DIM == 3) {
        if (ok && own) {
            const T* q0 = reinterpret_cast<const T*>(stage(0) + Lay::p_q);
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) qzp[i] = lds<T>(q0 + (j * DIM + 2) * qstride + qi);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bool alive = !__syncthreads_or(!ok);
    if (!alive && t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
    bool bad = false;
    int p_stop = z0 - 1;
    for (int p = z0; p < z1 && alive; ++p) {
        const int s = p - z0 + 1;
        const int cs = s % 3, ps = (s + 2) % 3;
        // stage ps held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 < z1) issue(p + 2, ps, false);
        ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        const unsigned char* st = stage(cs);
        const T* uS = reinterpret_cast<const T*>(st + Lay::p_u);
        const float* dS = reinterpret_cast<const float*>(st + Lay::p_d);
        const T* qS = reinterpret_cast<const T*>(st + Lay::p_q);
        float u[HL], d[HL];
        float mloc = 3.0e38f;
#pragma unroll
        for (int i = 0; i < HL; ++i) {
            const int j = half_label(h, i);
            u[i] = 0.f;
            d[i] = 0.f;
            if (own && (EXACT || j < nl)) {
                u[i] = lds<T>(uS + j * tile + v);
                const T* qx = qS + (j * DIM + 0) * qstride + qi;
                const T* qy = qS + (j * DIM + 1) * qstride + qi;
                float dv = (lds<T>(qx) - lds<T>(qx - 1)) + (lds<T>(qy) - lds<T>(qy - Lay::QBX));
                if constexpr (DIM == 3) {
                    const float qz = lds<T>(qS + (j * DIM + 2) * qstride + qi);
                    dv += qz - qzp[i];
                    qzp[i] = qz;
                }
                d[i] = dS[j * tile + v] + dv;
                mloc = fminf(mloc, d[i]);
            }
        }
        const float m = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
        float sloc = 0.f;
#pragma unroll
        for (int i = 0; i < HL; ++i) {
            const int j = half_label(h, i);
            if (own && (EXACT || j < nl)) {
                u[i] *= ex2_approx((d[i] - m) * kexp);
                sloc += u[i];
            }
        }
        const float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
        if (own) {
            if (!((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
            const float inv = rcp_fast(sum);
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) stu<T>(slot_ptr<IDX32>(u_out, j, p, n, plane, vox), u[i] * inv);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        p_stop = p;
        if (__syncthreads_or(!ok)) alive = false;
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    if (!alive && t == 0) {
        // bounded drain: the plane whose wait gave up and every plane issued after it
        const int hi = min(p_stop + 2, z1 - 1);
        for (int p = p_stop; p <= hi; ++p) {
            const int s = p - z0 + 1;
            mbar_wait_bounded(bar0 + 8 * (s % 3), (unsigned)((s / 3) & 1));
        }
    }
}

// Flow sweep on the labelling the prox sweep just wrote.  Plane p of the
// chunk (and the halo plane z1 inside the grid) lives in stage (p - z0) % 3;
// the flow step of plane p-1 runs at step p with its x / y steps, u, q and S
// carried in registers and the z difference from plane p's u.
template <int MAXL, int DIM, typename T, bool EXACT, bool IDX32>
__global__ void __launch_bounds__(INPLACE_TMA_NT, 1)
flow_inplace_tma_kernel(const StepArgs<MAXL, MAXL> a, const __grid_constant__ InplaceMaps maps) {
    constexpr int HL = MAXL / 2;
    using Lay = InplaceLayout<MAXL, DIM, T>;
    constexpr int ustride = TMA_UY * TMA_BX;
    constexpr int tile = Lay::tile;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x, h = t & 1, v = t >> 1;
    const int nl = EXACT ? MAXL : a.nl;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, a.nz);
    const int zl = min(z1, a.nz - 1);  // last plane read (the chunk's z halo, if inside the grid)
    const long long n = a.n, plane = (long long)a.px * a.ny;
    T* __restrict__ q_out = static_cast<T*>(a.q_out);
    const int has_S = a.S != nullptr;
    const unsigned bar0 = smem_addr(smem + Lay::f_bar);
    const unsigned bytes = (unsigned)(nl * ustride * sizeof(T)) + (unsigned)(DIM * nl * tile * sizeof(T)) +
                           (has_S ? (unsigned)(tile * 4) : 0u);
    auto stage = [&](int k) { return smem + k * Lay::f_stage; };
    auto issue = [&](int p, int k) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage(k);
        mbar_expect_tx(bar, bytes);
        tma_load_4d(smem_addr(st + Lay::f_u), &maps.u_halo, x0, y0, p, 0, bar);
        tma_load_4d(smem_addr(st + Lay::f_q), &maps.q_tile, x0, y0, p, 0, bar);
        if (has_S) tma_load_3d(smem_addr(st + Lay::f_s), &maps.S, x0, y0, p, bar);
    };
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(z0, 0);
        if (z0 + 1 <= zl) issue(z0 + 1, 1);
    }
    __syncthreads();
    const int ex = v & (FTX - 1), ey = v / FTX;
    const int xe = x0 + ex, ye = y0 + ey;
    const bool own = xe < a.nx && ye < a.ny;
    const int ui = ey * TMA_BX + ex;
    const long long vox = (long long)ye * a.px + xe;
    // zero steps at the last index (u beyond the grid is zero-filled by the box)
    const float cx = xe < a.nx - 1 ? a.ctau : 0.f;
    const float cy = ye < a.ny - 1 ? a.ctau : 0.f;
    float cap[HL];
#pragma unroll
    for (int i = 0; i < HL; ++i) cap[i] = a.s_node[half_label(h, i)];
    float gxp[HL], gyp[HL], up[HL], qxp[HL], qyp[HL], qzp[HL];
#pragma unroll
    for (int i = 0; i < HL; ++i) gxp[i] = gyp[i] = up[i] = qxp[i] = qyp[i] = qzp[i] = 0.f;
    float sprev = 1.0f;
    bool alive = true;
    int p_stop = z0;
    for (int p = z0; p <= z1 && alive; ++p) {
        const int s = p - z0;
        const int cs = s % 3, ns = (s + 2) % 3;
        // stage ns held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 <= zl) issue(p + 2, ns);
        bool ok = true;
        if (p <= zl) ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        const unsigned char* st = stage(cs);
        const T* uS = reinterpret_cast<const T*>(st + Lay::f_u);
        const T* qS = reinterpret_cast<const T*>(st + Lay::f_q);
        float uc[HL];
#pragma unroll
        for (int i = 0; i < HL; ++i) uc[i] = 0.f;
        if (own && p <= zl) {
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) uc[i] = lds<T>(uS + j * ustride + ui);
            }
        }
        // flow step of plane p-1
        if (own && p > z0) {
            const int pm = p - 1;
            const float cz = pm < a.nz - 1 ? a.ctau : 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) {
                    float yv[DIM];
                    yv[0] = qxp[i] - gxp[i];
                    yv[1] = qyp[i] - gyp[i];
                    if constexpr (DIM == 3) yv[2] = qzp[i] - cz * (uc[i] - up[i]);
                    project_nb<DIM>(yv, cap[i] * sprev, a.aniso);
#pragma unroll
                    for (int k = 0; k < DIM; ++k)
                        stv<T>(slot_ptr<IDX32>(q_out, j * DIM + k, pm, n, plane, vox), yv[k]);
                }
            }
        }
        // this plane's x / y steps, u, q and S for the next step
        if (own && p < z1) {
            sprev = has_S ? reinterpret_cast<const float*>(st + Lay::f_s)[v] : 1.0f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) {
                    const T* uj = uS + j * ustride + ui;
                    gxp[i] = cx * (lds<T>(uj + 1) - uc[i]);
                    gyp[i] = cy * (lds<T>(uj + TMA_BX) - uc[i]);
                    up[i] = uc[i];
                    qxp[i] = lds<T>(qS + (j * DIM + 0) * tile + v);
                    qyp[i] = lds<T>(qS + (j * DIM + 1) * tile + v);
                    if constexpr (DIM == 3) qzp[i] = lds<T>(qS + (j * DIM + 2) * tile + v);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        p_stop = p;
        if (__syncthreads_or(!ok)) alive = false;
    }
    if (!alive && t == 0) {
        // bounded drain: the plane whose wait gave up and every plane issued after it
        const int hi = min(p_stop + 2, zl);
        for (int p = p_stop; p <= hi; ++p) {
            const int s = p - z0;
            mbar_wait_bounded(bar0 + 8 * (s % 3), (unsigned)((s / 3) & 1));
        }
    }
}

}  // namespace pfm
