// pfm_tma.cuh -- TMA-pipelined fused iteration for the Potts model (sm_103a).
//
// Same arithmetic as fused_step_kernel (label prox of plane p on the
// halo-extended 33 x 9 tile, then the flow step of plane p-1), but every
// operand of a plane is brought into shared memory by the Tensor Memory
// Accelerator (cp.async.bulk.tensor) through a 3-stage ring guarded by
// mbarriers.  An iteration reads only its own plane's stage: what the flow
// step of plane p-1 needs at a voxel (its flows, g and S) stays in the
// registers of the threads that own the voxel, the neighbours' g goes
// through a two-plane shared buffer, so the stage of plane p-1 is refilled
// with plane p+2 at the start of plane p and two planes are in flight while
// one is consumed.  Out-of-range box elements (x0-4 < 0, y0-1 < 0, z = -1,
// beyond the far edges) are zero-filled by the TMA unit, which is exactly
// the zero boundary flow of the divergence.
//
// Every mbarrier wait is bounded by a cycle budget; on expiry the kernel
// sets FLAG_TIMEOUT, stops issuing, waits (bounded) for its own copies in
// flight and returns.
#pragma once

#include <cuda.h>

#include "pfm_device.cuh"

namespace pfm {

constexpr unsigned FLAG_TIMEOUT = 8u;

constexpr int TMA_BX = 40;       // u / D box width in x: x0 .. x0+39
constexpr int TMA_UY = FEY;      // 9 rows for u and D: y0 .. y0+8
constexpr int TMA_QY = FEY + 1;  // 10 rows for flows: y0-1 .. y0+8
constexpr int TMA_STAGES = 3;
constexpr long long TMA_WAIT_CYCLES = 4000000000ll;  // about 2 s at 2 GHz

template <int MAXL, int DIM, typename T>
struct TmaLayout {
    // the flow box starts QOFF elements left of the tile (a TMA box must
    // start on a 16-byte boundary) and spans x0-QOFF .. x0+FTX+QOFF-1
    static constexpr int QOFF = 16 / (int)sizeof(T);
    static constexpr int QBX = FTX + 2 * QOFF;
    static constexpr int u_elems = MAXL * TMA_UY * TMA_BX;
    static constexpr int q_elems = DIM * MAXL * TMA_QY * QBX;
    static constexpr int s_elems = FTY * FTX;
    static constexpr int align128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int u_off = 0;
    static constexpr int d_off = align128(u_off + u_elems * (int)sizeof(T));
    static constexpr int q_off = align128(d_off + u_elems * 4);
    static constexpr int s_off = align128(q_off + q_elems * (int)sizeof(T));
    static constexpr int stage_bytes = align128(s_off + s_elems * 4);
    // field g (what the flow step differentiates) of planes p-1 and p, FP32
    static constexpr int g_elems = MAXL * TMA_UY * TMA_BX;
    static constexpr int g_off = TMA_STAGES * stage_bytes;
    static constexpr int bar_off = align128(g_off + 2 * g_elems * 4);
    static constexpr int total_bytes = bar_off + 64 + 128;  // + slack to align the base to 128 B
};

// Staged flow box: coordinate 3 is node * DIM + component, as in the global
// layout q[node][comp][z][y][x].
struct TmaMaps {
    CUtensorMap u, q, D, S;  // u / q of the input buffers of this launch
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One arrival on a barrier (release: the thread's earlier shared-memory
// writes are visible to a thread whose wait on the phase succeeds).
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the budget (in clock cycles; every pipeline uses
// TMA_WAIT_CYCLES) ran out before the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity,
                                                  long long budget = TMA_WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

template <typename T> __device__ __forceinline__ float lds(const T* p);
template <> __device__ __forceinline__ float lds<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float lds<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float lds<__half>(const __half* p) { return __half2float(*p); }
template <typename T> __device__ __forceinline__ void sts(T* p, float v);
template <> __device__ __forceinline__ void sts<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void sts<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ void sts<__half>(__half* p, float v) { stv<__half>(p, v); }

// Two threads per voxel: thread pair (2v, 2v+1) shares voxel v, each owning
// half of the labels, J(h, i) = 4*(i/2) + 2*h + i%2 (halves {0,1,4,5} and
// {2,3,6,7}: the two lanes of a pair touch shared-memory banks 16 apart).
// The per-voxel minimum and normaliser of the prox are combined with one
// lane shuffle each; the flow step of a label needs nothing from the other
// half.  This doubles the resident warps (20 per SM) for the same staging.
constexpr int TMA_NT = 2 * FUSED_NT;  // 640 threads

__device__ __forceinline__ int half_label(int h, int i) { return 4 * (i >> 1) + 2 * h + (i & 1); }

// 2^x with the hardware approximation (relative error about 2^-22;
// subnormal results flush to zero, where the labelling is negligible anyway).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Pointer to slot (component c, plane p, voxel vox) of a pitched array with
// n slots per component and `plane` slots per plane.  IDX32: the launch
// guarantees every offset < 2^32, so the offset is formed in 32 bits and
// widened by the address computation itself (one wide multiply-add per
// access instead of a 64-bit multiply and add).
template <bool IDX32, typename T>
__device__ __forceinline__ T* slot_ptr(T* base, int c, int p, long long n, long long plane, long long vox) {
    if constexpr (IDX32)
        return base + ((unsigned)c * (unsigned)n + (unsigned)p * (unsigned)plane + (unsigned)vox);
    else
        return base + ((long long)c * n + (long long)p * plane + vox);
}

// 1/x by the hardware approximation (at most 1 ulp from the rounded
// quotient) for normal x; subnormal, zero and NaN x take the IEEE division.
__device__ __forceinline__ float rcp_fast(float x) {
    if (x >= 1.17549435e-38f) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    return 1.0f / x;
}

// 1/sqrt(x) by the hardware approximation (relative error below 2^-22);
// a subnormal x counts as 0 and gives +inf, which the projection maps to
// the unscaled vector (its length is far below any positive capacity).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Branch-free projection onto {|y| <= s} (s >= 0): scale min(1, s/|y|), with
// s = 0 mapping every y to 0.
template <int DIM>
__device__ __forceinline__ void project_nb(float (&y)[DIM], float s, int aniso) {
    if (aniso) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) y[k] = fminf(fmaxf(y[k], -s), s);
    } else {
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) r2 = fmaf(y[k], y[k], r2);
        const float f = s > 0.f ? fminf(1.0f, s * rsqrt_approx(r2)) : 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) y[k] *= f;
    }
}

// EXACT: the problem has exactly MAXL labels (no per-label guards).
// WITH_E: also accumulate the primal energy E(u) and the pseudo-flow dual
// P(q) of the INPUT state (u_in, q_in) of this iteration into one (E, P)
// partial per CTA: P of plane p from the prox's per-voxel minimum, E of
// plane p-1 (whose z-gradient needs plane p) during the flow phase.  The
// staged u is never overwritten, so its neighbours are still the input.
template <int MAXL, int DIM, typename T, bool EXACT, bool WITH_E, bool IDX32>
__global__ void __launch_bounds__(TMA_NT, 1)
fused_tma_kernel(const StepArgs<MAXL, MAXL> a, const __grid_constant__ TmaMaps maps, double* partial) {
    static_assert(MAXL % 4 == 0, "label halves need MAXL % 4 == 0");
    constexpr int HL = MAXL / 2;
    using Lay = TmaLayout<MAXL, DIM, T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ double sE[TMA_NT / 32], sP[TMA_NT / 32];
    // TMA destinations start on 128-byte boundaries
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x;
    const int h = t & 1;
    const int v = t >> 1;
    const int nl = EXACT ? MAXL : a.nl;
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
    const unsigned bytes_q = (unsigned)(DIM * nl * TMA_QY * Lay::QBX * sizeof(T));
    const unsigned bytes_s = has_S ? (unsigned)(FTX * FTY * 4) : 0u;
    const unsigned bar0 = smem_addr(smem + Lay::bar_off);
    const float kexp = -a.inv_c * 1.4426950408889634f;  // exp(-(d-m)/c) = 2^((d-m) kexp)
    constexpr int qstride = TMA_QY * Lay::QBX;
    constexpr int ustride = TMA_UY * TMA_BX;
    float* gbuf = reinterpret_cast<float*>(smem + Lay::g_off);

    auto stage_ptr = [&](int k) { return smem + k * Lay::stage_bytes; };
    // producer: bring plane p (full, or flows only) into stage k
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

    // An iteration reads only the stage of its own plane (what the flow step
    // and the energy of plane p-1 need at the voxel is kept in registers), so
    // the ring runs two planes ahead.
    int inflight_hi = z0;  // highest plane issued
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        issue(z0 - 1, 0, true);   // flows of plane z0-1 (zero-filled when z0 = 0)
        issue(z0, 1, false);
        if (z0 + 1 <= z1 && z0 + 1 < a.nz) {
            issue(z0 + 1, 2, false);
            inflight_hi = z0 + 1;
        }
    }
    __syncthreads();

    // Voxel of this thread pair on the halo-extended 33 x 9 tile, owned voxels
    // first (v < 256: the 32 x 8 tile, row-major), then the y-halo row (ey = 8)
    // and the x-halo column (ex = 32).  The same pair runs the prox of plane p
    // and the flow step of plane p-1 at its voxel, so the field g at its own
    // voxel (both planes) stays in registers and only the x+1 / y+1
    // neighbours' g goes through shared memory: one barrier per plane.
    const bool inE = v < FNE;
    const int ex = v < FTX * FTY ? (v & (FTX - 1)) : v < FTX * FTY + FTX ? v - FTX * FTY : FTX;
    const int ey = v < FTX * FTY ? v / FTX : v < FTX * FTY + FTX ? FTY : v - (FTX * FTY + FTX);
    const int xe = x0 + ex, ye = y0 + ey;
    const bool validE = inE && xe < a.nx && ye < a.ny;
    const bool ownerE = validE && v < FTX * FTY;
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * Lay::QBX + (ex + Lay::QOFF);
    const long long vox = (long long)ye * a.px + xe;  // slot of this voxel in its plane
    // forward differences are zero at the last index: zero steps there (the
    // g slots outside the grid hold zeros, so a zero step never meets a NaN)
    const float cx = xe < a.nx - 1 ? a.ctau : 0.f;
    const float cy = ye < a.ny - 1 ? a.ctau : 0.f;

    for (int k = t; k < 2 * Lay::g_elems; k += TMA_NT) gbuf[k] = 0.f;
    float cap[HL];  // per-label capacity factors of this thread's label half
#pragma unroll
    for (int i = 0; i < HL; ++i) cap[i] = a.s_node[half_label(h, i)];
    // this voxel's state carried from plane p-1 to plane p: g, the three flow
    // components (the z one also closes the divergence of plane p) and S
    float gprev[HL], gcur[HL], qxp[HL], qyp[HL], qzp[HL];
    float sprev = 1.0f;
#pragma unroll
    for (int i = 0; i < HL; ++i) gprev[i] = gcur[i] = qxp[i] = qyp[i] = qzp[i] = 0.f;
    // flows of plane z0-1 (z component only: its x / y flow steps belong to
    // the previous z-chunk)
    bool ok = mbar_wait_bounded(bar0, 0u);
    if constexpr (DIM == 3) {
        if (ok && validE) {
            const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + Lay::q_off);
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) qzp[i] = lds<T>(q0 + (j * DIM + 2) * qstride + qi);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        s_abort = 1;
    }
    // energy of the input state (WITH_E): the staged u at this voxel and the
    // x / y part of its gradient norm (|gx|+|gy| or gx^2+gy^2), carried to the
    // next plane, which supplies the z difference
    float uin_prev[HL], txy_prev[HL];
#pragma unroll
    for (int i = 0; i < HL; ++i) uin_prev[i] = txy_prev[i] = 0.f;
    bool bad = false;
    SumF sumE, sumP;
    int p_stop = z0 - 1;  // first plane whose stage may still be in flight at an abort
    for (int p = z0; p <= z1 && !s_abort; ++p) {
        const int s = p - z0 + 1;
        const int cs = s % 3, ps = (s + 2) % 3;
        // stage ps held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 <= z1 && p + 2 < a.nz) {
            issue(p + 2, ps, false);
            inflight_hi = p + 2;
        }
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + (p & 1) * Lay::g_elems;              // g of plane p (written now)
        const float* gP = gbuf + ((p + 1) & 1) * Lay::g_elems;  // g of plane p-1 (neighbours)
        // each thread waits for its stage itself; a timeout is raised to the
        // whole CTA at the end-of-plane barrier
        ok = true;
        if (p < a.nz) ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        float qxc[HL], qyc[HL], qzc[HL], uin[HL], txy[HL];
#pragma unroll
        for (int i = 0; i < HL; ++i) qxc[i] = qyc[i] = qzc[i] = uin[i] = txy[i] = 0.f;
        float scur = 1.0f;
        float eD = 0.f;  // sum of D u over this thread's labels of plane p (WITH_E)

        // ---- label prox of plane p on the halo-extended tile (uniform branch)
        if (p < a.nz) {
            const T* uS = reinterpret_cast<const T*>(cst + Lay::u_off);
            const float* dS = reinterpret_cast<const float*>(cst + Lay::d_off);
            const T* qS = reinterpret_cast<const T*>(cst + Lay::q_off);
            if (has_S && ownerE) scur = reinterpret_cast<const float*>(cst + Lay::s_off)[ey * FTX + ex];
            // Divergence without boundary tests: the normal flow component at
            // the last index of each axis is an invariant zero of the stored
            // state (zero at initialisation, kept by the flow step, enforced by
            // pfm_set_flows) and the box is zero-filled outside the grid.
            float u[HL], d[HL];
            float mloc = 3.0e38f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                u[i] = 0.f;
                d[i] = 0.f;
                if (validE && (EXACT || j < nl)) {
                    u[i] = lds<T>(uS + j * ustride + ui);
                    const T* qx = qS + (j * DIM + 0) * qstride + qi;
                    const T* qy = qS + (j * DIM + 1) * qstride + qi;
                    qxc[i] = lds<T>(qx);
                    qyc[i] = lds<T>(qy);
                    float dv = (qxc[i] - lds<T>(qx - 1)) + (qyc[i] - lds<T>(qy - Lay::QBX));
                    if constexpr (DIM == 3) {
                        qzc[i] = lds<T>(qS + (j * DIM + 2) * qstride + qi);
                        dv += qzc[i] - qzp[i];
                    }
                    const float Dv = dS[j * ustride + ui];
                    d[i] = Dv + dv;
                    mloc = fminf(mloc, d[i]);
                    if constexpr (WITH_E) {
                        uin[i] = u[i];
                        if (ownerE) {
                            const float gx = cx != 0.f ? lds<T>(uS + j * ustride + ui + 1) - u[i] : 0.f;
                            const float gy = cy != 0.f ? lds<T>(uS + j * ustride + ui + TMA_BX) - u[i] : 0.f;
                            txy[i] = a.aniso ? fabsf(gx) + fabsf(gy) : fmaf(gx, gx, gy * gy);
                            if (p < z1) eD = fmaf(Dv, u[i], eD);
                        }
                    }
                }
            }
            // per-voxel minimum over both halves: the dual term of this voxel,
            // and the exponent shift (NORMALISED only)
            const float dmin = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
            if constexpr (WITH_E) {
                if (ownerE && p < z1 && h == 0) sumP.add(dmin);
            }
            const float m = a.literal ? 0.f : dmin;
            float sloc = 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (validE && (EXACT || j < nl)) {
                    u[i] *= ex2_approx((d[i] - m) * kexp);
                    sloc += u[i];
                }
            }
            const float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
            if (validE) {
                if (!((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
                const float inv = rcp_fast(sum);
#pragma unroll
                for (int i = 0; i < HL; ++i) {
                    const int j = half_label(h, i);
                    if (EXACT || j < nl) {
                        const float un = u[i] * inv;
                        gcur[i] = a.literal ? u[i] : un;
                        gC[j * ustride + ui] = gcur[i];
                        if (ownerE && p < z1) stu<T>(slot_ptr<IDX32>(uout, j, p, n, plane, vox), un);
                    }
                }
            }
        }

        // ---- flow step of plane p-1 at the owned voxel (one label half per
        // thread): g of plane p-1 at x+1 and y+1 from the previous plane's
        // prox (visible since the last barrier), own g of planes p-1 and p
        // from registers
        const int pm = p - 1;
        if (pm >= z0 && ownerE) {
            const float sf = sprev;
            const float cz = pm < a.nz - 1 ? a.ctau : 0.f;
            float eloc = 0.f;
#pragma unroll
            for (int i = 0; i < HL; ++i) {
                const int j = half_label(h, i);
                if (EXACT || j < nl) {
                    const float* gj = gP + j * ustride;
                    const float g0 = gprev[i];
                    float yv[DIM];
                    yv[0] = qxp[i] - cx * (gj[ui + 1] - g0);
                    yv[1] = qyp[i] - cy * (gj[ui + TMA_BX] - g0);
                    if constexpr (DIM == 3) yv[2] = qzp[i] - cz * (gcur[i] - g0);
                    const float sj = cap[i] * sf;
                    if constexpr (WITH_E) {
                        // TV term of plane p-1 on the input labelling: x / y part
                        // from the previous plane, z difference with this plane's
                        // staged u
                        float gz = 0.f;
                        if constexpr (DIM == 3) gz = cz != 0.f ? uin[i] - uin_prev[i] : 0.f;
                        const float nv = a.aniso ? txy_prev[i] + fabsf(gz) : sqrt_approx(fmaf(gz, gz, txy_prev[i]));
                        eloc = fmaf(sj, nv, eloc);
                    }
                    project_nb<DIM>(yv, sj, a.aniso);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) stv<T>(slot_ptr<IDX32>(qout, j * DIM + k, pm, n, plane, vox), yv[k]);
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
            uin_prev[i] = uin[i];
            txy_prev[i] = txy[i];
        }
        sprev = scur;
        // order this plane's shared-memory accesses before the TMA that
        // refills a stage at the next step; one barrier per plane, which also
        // carries a timed-out wait of any thread to the whole CTA
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        p_stop = p;
        if (__syncthreads_or(!ok)) {
            if (t == 0) s_abort = 1;
            break;
        }
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    if (s_abort && t == 0) {
        // bounded drain of this CTA's copies that may still be in flight: the
        // plane whose wait gave up and every plane issued after it (planes
        // consumed earlier are complete and their stages may have been refilled)
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

// ---------------------------------------------------------------------------
// TMA-staged energy / dual of a Potts state (same boxes and maps as the
// iteration).  Each CTA owns a 32 x 8 tile of a z-chunk; plane r needs u of
// plane r+1 (z-gradient), so planes r+1 and r+2 are in flight while r is
// summed; the own voxel's z-flow of plane r-1 (divergence) is carried in
// registers.  Four threads per voxel (lane 4k+h takes labels h, h+4, ...),
// the per-voxel minimum of the dual combined by two lane shuffles.  One
// (E, P) partial per CTA, FP64 accumulation.
// ---------------------------------------------------------------------------
constexpr int ENERGY_TMA_NT = 4 * FTX * FTY;  // 1024 threads

template <int MAXL, int DIM, typename T>
__global__ void __launch_bounds__(ENERGY_TMA_NT, 1)
energy_tma_kernel(const StepArgs<MAXL, MAXL> a, const __grid_constant__ TmaMaps maps, double* partial) {
    static_assert(MAXL % 4 == 0, "labels are split in four");
    constexpr int QL = MAXL / 4;
    using Lay = TmaLayout<MAXL, DIM, T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ double sE[ENERGY_TMA_NT / 32], sP[ENERGY_TMA_NT / 32];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x;
    const int h = t & 3;
    const int v = t >> 2;
    const int nl = a.nl;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, a.nz);
    const long long n = a.n;
    const long long plane = (long long)a.px * a.ny;
    const int has_S = a.S != nullptr;
    const unsigned bytes = (unsigned)(nl * TMA_UY * TMA_BX * sizeof(T)) + (unsigned)(nl * TMA_UY * TMA_BX * 4) +
                           (unsigned)(DIM * nl * TMA_QY * Lay::QBX * sizeof(T)) +
                           (has_S ? (unsigned)(FTX * FTY * 4) : 0u);
    const unsigned bar0 = smem_addr(smem + Lay::bar_off);
    constexpr int qstride = TMA_QY * Lay::QBX;
    constexpr int ustride = TMA_UY * TMA_BX;
    auto stage_ptr = [&](int k) { return smem + k * Lay::stage_bytes; };
    auto issue = [&](int p, int k) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage_ptr(k);
        mbar_expect_tx(bar, bytes);
        tma_load_4d(smem_addr(st + Lay::q_off), &maps.q, x0 - Lay::QOFF, y0 - 1, p, 0, bar);
        tma_load_4d(smem_addr(st + Lay::u_off), &maps.u, x0, y0, p, 0, bar);
        tma_load_4d(smem_addr(st + Lay::d_off), &maps.D, x0, y0, p, 0, bar);
        if (has_S) tma_load_3d(smem_addr(st + Lay::s_off), &maps.S, x0, y0, p, bar);
    };
    int issued_hi = z0;
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        issue(z0, 0);
        if (z0 + 1 < a.nz) {
            issue(z0 + 1, 1);
            issued_hi = z0 + 1;
        }
    }
    __syncthreads();
    const int mx = v % FTX, my = v / FTX;
    const int x = x0 + mx, y = y0 + my;
    const bool own = x < a.nx && y < a.ny;
    float qzp[QL];  // own z-flow of plane r-1 for this thread's labels
#pragma unroll
    for (int i = 0; i < QL; ++i) qzp[i] = 0.f;
    if constexpr (DIM == 3) {
        if (own && z0 > 0) {
            const T* qin = static_cast<const T*>(a.q_in);
            const long long i0 = (long long)(z0 - 1) * plane + (long long)y * a.px + x;
#pragma unroll
            for (int i = 0; i < QL; ++i) {
                const int j = h + 4 * i;
                if (j < nl) qzp[i] = ldv<T>(qin + ((long long)j * DIM + 2) * n + i0);
            }
        }
    }
    SumF sumE, sumP;
    int r_stop = z0;  // first plane whose stage may still be in flight at an abort
    for (int r = z0; r < z1; ++r) {
        const int s = r - z0;
        const int cs = s % 3, n1 = (s + 1) % 3, n2 = (s + 2) % 3;
        if (t == 0 && r + 2 <= z1 && r + 2 < a.nz) {
            issue(r + 2, n2);
            issued_hi = r + 2;
        }
        bool ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (ok && r + 1 < a.nz) ok = mbar_wait_bounded(bar0 + 8 * n1, (unsigned)(((s + 1) / 3) & 1));
        if (!ok) {
            atomicOr(a.flags, FLAG_TIMEOUT);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        float eData = 0.f, tv = 0.f, dmin = 3.0e38f;
        if (own) {
            const unsigned char* cst = stage_ptr(cs);
            const unsigned char* nst = stage_ptr(n1);
            const T* uS = reinterpret_cast<const T*>(cst + Lay::u_off);
            const T* uN = reinterpret_cast<const T*>(nst + Lay::u_off);
            const float* dS = reinterpret_cast<const float*>(cst + Lay::d_off);
            const T* qS = reinterpret_cast<const T*>(cst + Lay::q_off);
            const float* sS = reinterpret_cast<const float*>(cst + Lay::s_off);
            const int ui = my * TMA_BX + mx;
            const int qi = (my + 1) * Lay::QBX + (mx + Lay::QOFF);
            const float sf = has_S ? sS[my * FTX + mx] : 1.0f;
#pragma unroll
            for (int i = 0; i < QL; ++i) {
                const int j = h + 4 * i;
                if (j < nl) {
                    const T* uj = uS + j * ustride;
                    const float u0 = lds<T>(uj + ui);
                    const float Dj = dS[j * ustride + ui];
                    eData = fmaf(Dj, u0, eData);
                    float gr[DIM];
                    gr[0] = x < a.nx - 1 ? lds<T>(uj + ui + 1) - u0 : 0.f;
                    gr[1] = y < a.ny - 1 ? lds<T>(uj + ui + TMA_BX) - u0 : 0.f;
                    if constexpr (DIM == 3)
                        gr[2] = r < a.nz - 1 ? lds<T>(uN + j * ustride + ui) - u0 : 0.f;
                    float nv;
                    if (a.aniso) {
                        nv = 0.f;
#pragma unroll
                        for (int k = 0; k < DIM; ++k) nv += fabsf(gr[k]);
                    } else {
                        float r2 = 0.f;
#pragma unroll
                        for (int k = 0; k < DIM; ++k) r2 = fmaf(gr[k], gr[k], r2);
                        nv = sqrt_approx(r2);
                    }
                    tv = fmaf(a.s_node[j] * sf, nv, tv);
                    const T* qx = qS + (j * DIM + 0) * qstride;
                    const T* qy = qS + (j * DIM + 1) * qstride;
                    float dv = (x < a.nx - 1 ? lds<T>(qx + qi) : 0.f) - lds<T>(qx + qi - 1);
                    dv += (y < a.ny - 1 ? lds<T>(qy + qi) : 0.f) - lds<T>(qy + qi - Lay::QBX);
                    if constexpr (DIM == 3) {
                        const float qz = lds<T>(qS + (j * DIM + 2) * qstride + qi);
                        dv += (r < a.nz - 1 ? qz : 0.f) - qzp[i];
                        qzp[i] = qz;
                    }
                    dmin = fminf(dmin, Dj + dv);
                }
            }
        }
        // minimum over the voxel's four label groups (lanes 4k .. 4k+3)
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
        for (int k = 0; k < ENERGY_TMA_NT / 32; ++k) {
            E += sE[k];
            P += sP[k];
        }
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partial[2 * b] = E;
        partial[2 * b + 1] = P;
    }
}

}  // namespace pfm
