// pfm_tma_ishikawa.cuh -- TMA-pipelined fused iteration of the Ishikawa
// model (Algorithm 3): N levels, N+1 ordered labels L_0..L_N, one flow per
// level.
//
// Per voxel, with e_k the divergence of level k's flow:
//   d_{L_i} = D_{L_i} + e_1 + ... + e_i          (cumulative excess, top-down)
//   u <- u e^{-(d - m)/c} / sum                  (prox and normalisation)
//   g_i = u_{L_i} + ... + u_{L_N}                (bottom-up accumulation)
//   q_i <- Proj_{|.| <= S_i}(q_i - c tau grad g_i), i = 1..N
// The kernel is the Potts kernel's plane pipeline (32 x 8 tiles, three-stage
// cp.async.bulk.tensor ring, two planes in flight, one barrier per plane,
// flows / g / S of the voxel carried in registers) with the two threads of a
// voxel owning CONTIGUOUS label halves: thread 0 labels 0..3 with the flows
// of levels 1..3, thread 1 labels 4..7 with levels 4..7.  The prefix sums of
// the excess and the suffix sums of g are then the thread's own running sums
// plus one lane shuffle carrying the other half's total.
//
// Problem form: a label DAG whose flow-carrying nodes 0..N-1 are the levels
// (node k-1 is level k) with path weights W_(node k-1, L_j) = [j >= k], and
// whose other nodes carry no flow -- the chain S -> A_1 -> ... -> A_N with
// L_0 under S and L_i under A_i.  The solver detects it from the weights.
#pragma once

#include "pfm_tma.cuh"

namespace pfm {

constexpr int ISH_MAXL = 8;  // labels (N + 1 <= 8, N <= 7 levels)

// WITH_E: also reduce E(u) and P(q) of the input state into one (E, P)
// partial per CTA: P of plane p from the prox's per-voxel minimum; E of
// plane p-1 in the flow phase, the data term and, per level, S_k |grad g_k|
// of the input labelling's accumulated g_k = u_{L_k} + ... + u_{L_N} (the
// labels carry no capacity), its z-difference from plane p's staged u.  The
// update itself is the same arithmetic.
template <int MAXL, int MAXN, typename T, bool WITH_E, bool IDX32>
__global__ void __launch_bounds__(TMA_NT, 1)
ishikawa_tma_kernel(const StepArgs<MAXL, MAXN> a, const __grid_constant__ TmaMaps maps, double* partial) {
    constexpr int DIM = 3;
    constexpr int HL = ISH_MAXL / 2;
    using Lay = TmaLayout<ISH_MAXL, DIM, T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ double sE[TMA_NT / 32], sP[TMA_NT / 32];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x;
    const int h = t & 1;
    const int v = t >> 1;
    const int nl = a.nl;       // N + 1 labels
    const int nlev = nl - 1;   // N levels = flow-carrying nodes 0..N-1
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, a.nz);
    const long long n = a.n;
    const long long plane = (long long)a.px * a.ny;
    T* __restrict__ uout = static_cast<T*>(a.u_out);
    T* __restrict__ qout = static_cast<T*>(a.q_out);
    const int has_S = a.S != nullptr;
    const unsigned bytes_u = (unsigned)(nl * TMA_UY * TMA_BX * sizeof(T));
    const unsigned bytes_d = (unsigned)(nl * TMA_UY * TMA_BX * 4);
    const unsigned bytes_q = (unsigned)(DIM * nlev * TMA_QY * Lay::QBX * sizeof(T));
    const unsigned bytes_s = has_S ? (unsigned)(FTX * FTY * 4) : 0u;
    const unsigned bar0 = smem_addr(smem + Lay::bar_off);
    const float kexp = -a.inv_c * 1.4426950408889634f;  // exp(-(d-m)/c) = 2^((d-m) kexp)
    constexpr int qstride = TMA_QY * Lay::QBX;
    constexpr int ustride = TMA_UY * TMA_BX;
    float* gbuf = reinterpret_cast<float*>(smem + Lay::g_off);

    auto stage_ptr = [&](int k) { return smem + k * Lay::stage_bytes; };
    auto issue = [&](int p, int k, bool flows_only) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage_ptr(k);
        mbar_expect_tx(bar, flows_only ? bytes_q : bytes_u + bytes_d + bytes_q + bytes_s);
        tma_load_4d(smem_addr(st + Lay::q_off), &maps.q, x0 - Lay::QOFF, y0 - 1, p, 0, bar);
        if (!flows_only) {
            tma_load_4d(smem_addr(st + Lay::u_off), &maps.u, x0, y0, p, 0, bar);
            tma_load_4d(smem_addr(st + Lay::d_off), &maps.D, x0, y0, p, 0, bar);
            if (has_S) tma_load_3d(smem_addr(st + Lay::s_off), &maps.S, x0, y0, p, bar);
        }
    };

    int inflight_hi = z0;
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        issue(z0 - 1, 0, true);
        issue(z0, 1, false);
        if (z0 + 1 <= z1 && z0 + 1 < a.nz) {
            issue(z0 + 1, 2, false);
            inflight_hi = z0 + 1;
        }
    }
    __syncthreads();

    // voxel of this thread pair on the halo-extended 33 x 9 tile (owned first)
    const bool inE = v < FNE;
    const int ex = v < FTX * FTY ? (v & (FTX - 1)) : v < FTX * FTY + FTX ? v - FTX * FTY : FTX;
    const int ey = v < FTX * FTY ? v / FTX : v < FTX * FTY + FTX ? FTY : v - (FTX * FTY + FTX);
    const int xe = x0 + ex, ye = y0 + ey;
    const bool validE = inE && xe < a.nx && ye < a.ny;
    const bool ownerE = validE && v < FTX * FTY;
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * Lay::QBX + (ex + Lay::QOFF);
    const long long vox = (long long)ye * a.px + xe;
    const float cx = xe < a.nx - 1 ? a.ctau : 0.f;
    const float cy = ye < a.ny - 1 ? a.ctau : 0.f;

    for (int k = t; k < 2 * Lay::g_elems; k += TMA_NT) gbuf[k] = 0.f;
    // label j = HL*h + i of this thread; level j >= 1 has the flow of node j-1
    float cap[HL];
#pragma unroll
    for (int i = 0; i < HL; ++i) {
        const int j = HL * h + i;
        cap[i] = (j >= 1 && j <= nlev) ? a.s_node[j - 1] : 0.f;
    }
    float gprev[HL], gcur[HL], qxp[HL], qyp[HL], qzp[HL];
    float sprev = 1.0f;
#pragma unroll
    for (int i = 0; i < HL; ++i) gprev[i] = gcur[i] = qxp[i] = qyp[i] = qzp[i] = 0.f;
    bool ok = mbar_wait_bounded(bar0, 0u);
    if (ok && validE) {
        const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + Lay::q_off);
#pragma unroll
        for (int i = 0; i < HL; ++i) {
            const int j = HL * h + i;
            if (j >= 1 && j <= nlev) qzp[i] = lds<T>(q0 + ((j - 1) * DIM + 2) * qstride + qi);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        s_abort = 1;
    }
    // WITH_E: the input's accumulated g of each level at this voxel and the
    // x / y part of its gradient norm, carried to the next plane
    float ginp[HL], txy_prev[HL];
#pragma unroll
    for (int i = 0; i < HL; ++i) ginp[i] = txy_prev[i] = 0.f;
    SumF sumE, sumP;
    bool bad = false;
    int p_stop = z0 - 1;
    for (int p = z0; p <= z1 && !s_abort; ++p) {
        const int s = p - z0 + 1;
        const int cs = s % 3, ps = (s + 2) % 3;
        if (t == 0 && p + 2 <= z1 && p + 2 < a.nz) {
            issue(p + 2, ps, false);
            inflight_hi = p + 2;
        }
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + (p & 1) * Lay::g_elems;
        const float* gP = gbuf + ((p + 1) & 1) * Lay::g_elems;
        ok = true;
        if (p < a.nz) ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        float qxc[HL], qyc[HL], qzc[HL], gin[HL], txy[HL];
#pragma unroll
        for (int i = 0; i < HL; ++i) qxc[i] = qyc[i] = qzc[i] = gin[i] = txy[i] = 0.f;
        float scur = 1.0f;
        float eD = 0.f;  // sum of D u over this thread's labels of plane p (WITH_E)

        // ---- label prox of plane p on the halo-extended tile
        if (p < a.nz) {
            const T* uS = reinterpret_cast<const T*>(cst + Lay::u_off);
            const float* dS = reinterpret_cast<const float*>(cst + Lay::d_off);
            const T* qS = reinterpret_cast<const T*>(cst + Lay::q_off);
            if (has_S && ownerE) scur = reinterpret_cast<const float*>(cst + Lay::s_off)[ey * FTX + ex];
            // divergence of this half's levels and its running (prefix) sum
            float pre[HL];
            float run = 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = HL * h + i;
                if (validE && j >= 1 && j <= nlev) {
                    const T* qx = qS + ((j - 1) * DIM + 0) * qstride + qi;
                    const T* qy = qS + ((j - 1) * DIM + 1) * qstride + qi;
                    qxc[i] = lds<T>(qx);
                    qyc[i] = lds<T>(qy);
                    qzc[i] = lds<T>(qS + ((j - 1) * DIM + 2) * qstride + qi);
                    run += (qxc[i] - lds<T>(qx - 1)) + (qyc[i] - lds<T>(qy - Lay::QBX)) + (qzc[i] - qzp[i]);
                }
                pre[i] = run;
            }
            // the upper half adds the lower half's total excess
            const float lower = __shfl_xor_sync(0xffffffffu, run, 1);
            const float carry = h == 1 ? lower : 0.f;
            float u[HL], d[HL];
            float mloc = 3.0e38f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = HL * h + i;
                u[i] = 0.f;
                d[i] = 0.f;
                if (validE && j < nl) {
                    u[i] = lds<T>(uS + j * ustride + ui);
                    d[i] = dS[j * ustride + ui] + (pre[i] + carry);
                    mloc = fminf(mloc, d[i]);
                }
            }
            const float dmin = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
            if constexpr (WITH_E) {
                if (ownerE && p < z1 && h == 0) sumP.add(dmin);
                // input labelling: running suffix sums at x, x+1, y+1 of this
                // half, the lower half adding the upper half's totals
                float f0[HL], f1[HL], f2[HL];
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int i = HL - 1; i >= 0; --i) {
                    const int j = HL * h + i;
                    if (validE && j < nl) {
                        const T* uj = uS + j * ustride + ui;
                        s0 += u[i];
                        if (ownerE) {
                            s1 += lds<T>(uj + 1);
                            s2 += lds<T>(uj + TMA_BX);
                            if (p < z1) eD = fmaf(dS[j * ustride + ui], u[i], eD);
                        }
                    }
                    f0[i] = s0;
                    f1[i] = s1;
                    f2[i] = s2;
                }
                const float t0 = __shfl_xor_sync(0xffffffffu, s0, 1);
                const float t1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                const float t2 = __shfl_xor_sync(0xffffffffu, s2, 1);
                const float c0 = h == 0 ? t0 : 0.f, c1 = h == 0 ? t1 : 0.f, c2 = h == 0 ? t2 : 0.f;
#pragma unroll
                for (int i = 0; i < HL; ++i) {
                    const int j = HL * h + i;
                    if (j >= 1 && j <= nlev) {
                        gin[i] = f0[i] + c0;
                        const float gx = cx != 0.f ? (f1[i] + c1) - gin[i] : 0.f;
                        const float gy = cy != 0.f ? (f2[i] + c2) - gin[i] : 0.f;
                        txy[i] = a.aniso ? fabsf(gx) + fabsf(gy) : fmaf(gx, gx, gy * gy);
                    }
                }
            }
            const float m = a.literal ? 0.f : dmin;
            float sloc = 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = HL * h + i;
                if (validE && j < nl) {
                    u[i] *= ex2_approx((d[i] - m) * kexp);
                    sloc += u[i];
                }
            }
            const float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
            const float inv = rcp_fast(sum);
            if (validE && !((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
            // g of this half (normalised or, PAPER_LITERAL, unnormalised u)
            // and its running suffix sum; the lower half adds the upper
            // half's total
            float gl[HL];
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = HL * h + i;
                gl[i] = (validE && j < nl) ? (a.literal ? u[i] : u[i] * inv) : 0.f;
            }
            float suf[HL];
            float rs = 0.f;
#pragma unroll
            for (int i = HL - 1; i >= 0; --i) {
                rs += gl[i];
                suf[i] = rs;
            }
            const float upper = __shfl_xor_sync(0xffffffffu, rs, 1);
            const float gcarry = h == 0 ? upper : 0.f;
            if (validE) {
#pragma unroll
                for (int i = 0; i < HL; ++i) {
                    const int j = HL * h + i;
                    if (j < nl) {
                        if (ownerE && p < z1) stu<T>(slot_ptr<IDX32>(uout, j, p, n, plane, vox), u[i] * inv);
                        if (j >= 1) {
                            gcur[i] = suf[i] + gcarry;  // g of level j: labels j..N
                            gC[j * ustride + ui] = gcur[i];
                        }
                    }
                }
            }
        }

        // ---- flow step of plane p-1 at the owned voxel (levels of this half)
        const int pm = p - 1;
        if (pm >= z0 && ownerE) {
            const float sf = sprev;
            const float cz = pm < a.nz - 1 ? a.ctau : 0.f;
            float eloc = 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = HL * h + i;
                if (j >= 1 && j <= nlev) {
                    if constexpr (WITH_E) {
                        // TV of level j on the input labelling, plane p-1
                        const float gz = cz != 0.f ? gin[i] - ginp[i] : 0.f;
                        const float nv = a.aniso ? txy_prev[i] + fabsf(gz) : sqrt_approx(fmaf(gz, gz, txy_prev[i]));
                        eloc = fmaf(cap[i] * sf, nv, eloc);
                    }
                    const float* gj = gP + j * ustride;
                    const float g0 = gprev[i];
                    float yv[DIM];
                    yv[0] = qxp[i] - cx * (gj[ui + 1] - g0);
                    yv[1] = qyp[i] - cy * (gj[ui + TMA_BX] - g0);
                    yv[2] = qzp[i] - cz * (gcur[i] - g0);
                    project_nb<DIM>(yv, cap[i] * sf, a.aniso);
#pragma unroll
                    for (int k = 0; k < DIM; ++k)
                        stv<T>(slot_ptr<IDX32>(qout, (j - 1) * DIM + k, pm, n, plane, vox), yv[k]);
                }
            }
            if constexpr (WITH_E) sumE.add(eloc);
        }
        if constexpr (WITH_E) sumE.add(eD);
#pragma unroll
        for (int i = 0; i < HL; ++i) {
            gprev[i] = gcur[i];
            qxp[i] = qxc[i];
            qyp[i] = qyc[i];
            qzp[i] = qzc[i];
            ginp[i] = gin[i];
            txy_prev[i] = txy[i];
        }
        sprev = scur;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        p_stop = p;
        if (__syncthreads_or(!ok)) {
            if (t == 0) s_abort = 1;
            break;
        }
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    if (s_abort && t == 0) {
        for (int p = p_stop; p <= inflight_hi; ++p) {
            const int s = p - z0 + 1;
            mbar_wait_bounded(bar0 + 8 * (s % 3), (unsigned)((s / 3) & 1));
        }
    }
    if constexpr (WITH_E) {
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
            for (int k = 0; k < TMA_NT / 32; ++k) {
                E += sE[k];
                P += sP[k];
            }
            const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            partial[2 * b] = E;
            partial[2 * b + 1] = P;
        }
    }
}

}  // namespace pfm
