// pfm_tma_x2.cuh -- TMA-pipelined fused Potts iteration, two x-adjacent
// voxels per thread with packed FP32 pair arithmetic (sm_100+ f32x2).
//
// Same plane pipeline, staging boxes and shared-memory layout as
// fused_tma_kernel (Algorithm 1, one iteration: label prox of plane p on the
// halo-extended 33 x 9 tile, flow step of plane p-1 at the owned voxels),
// but a thread holds a voxel PAIR (x, x+1) and a quarter of the labels:
// lane h of the pair's four threads takes labels h, h+4, ...  Every load,
// every add / multiply / fused multiply-add and every store of the
// iteration then serves two voxels (64-bit shared loads and global stores of
// FP32 pairs, 32-bit ones of BF16 / F16 pairs; packed f32x2 add / multiply /
// fma),
// so the kernel issues fewer instructions per voxel-label update than the
// one-voxel-per-thread form (about a fifth fewer with BF16 storage: widening
// BF16 pairs, the per-voxel work below and the operands assembled from
// neighbours stay).  Only the hardware approximations (ex2, rsqrt, rcp),
// the minimum and the projection's scale stay per voxel.  The per-voxel
// minimum and normaliser of the prox are combined over the four lanes with
// two shuffle rounds.  Used for 16-bit storage: with FP32 storage the
// one-voxel kernel already runs at the bandwidth roof and this one measured
// slower.
//
// The halo-extended tile is covered by 153 pairs: 16 x 8 owned pairs, the
// 16 pairs of the y-halo row and 9 pairs (x0+32, x0+33) of the x-halo column,
// whose second voxel only pads the pair (it is computed from the staged box,
// never stored, never read).  A pair whose second voxel lies beyond the
// grid's last index computes it as zero and stores the pair into the row
// padding (the launch requires an even row pitch).
#pragma once

#include "pfm_tma.cuh"

namespace pfm {

constexpr int X2_PAIRS = (FTX / 2) * FTY + FTX / 2 + FEY;  // 128 + 16 + 9 = 153
constexpr int X2_NT = ((4 * X2_PAIRS + 31) / 32) * 32;      // 640 threads

// Shared memory of the pair kernel: the staging boxes of TmaLayout in a ring
// of four stages, four FP32 g planes, and one barrier per stage and per g
// plane (211.6 KB for 8 labels in 16-bit storage).
template <int MAXL, typename T>
struct X2Layout {
    using B = TmaLayout<MAXL, 3, T>;
    static constexpr int STAGES = 4;
    static constexpr int GBUF = 4;
    static constexpr int QBX = B::QBX, QOFF = B::QOFF;
    static constexpr int u_off = B::u_off, d_off = B::d_off, q_off = B::q_off, s_off = B::s_off;
    static constexpr int stage_bytes = B::stage_bytes;
    static constexpr int g_elems = B::g_elems;
    static constexpr int g_off = STAGES * stage_bytes;
    static constexpr int bar_off = B::align128(g_off + GBUF * g_elems * 4);
    static constexpr int total_bytes = bar_off + 8 * (STAGES + GBUF) + 128;
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// voxel pair (x, x+1) of a staged row; the pair starts at an even element
template <typename T> __device__ __forceinline__ float2 lds2(const T* p);
template <> __device__ __forceinline__ float2 lds2<float>(const float* p) {
    return *reinterpret_cast<const float2*>(p);
}
template <> __device__ __forceinline__ float2 lds2<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned w = *reinterpret_cast<const unsigned*>(p);
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> __device__ __forceinline__ float2 lds2<__half>(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
}
template <typename T> __device__ __forceinline__ void stv2(T* p, float2 v);
template <> __device__ __forceinline__ void stv2<float>(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
template <> __device__ __forceinline__ void stv2<__nv_bfloat16>(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
}
// F16 pairs: one conversion that rounds to nearest and saturates to
// +-65504 (a NaN stays NaN)
template <> __device__ __forceinline__ void stv2<__half>(__half* p, float2 v) {
    unsigned w;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(v.y), "f"(v.x));
    *reinterpret_cast<unsigned*>(p) = w;
}
// A labelling pair (the F16 floor of stu applies), stored as a pair even
// when its second voxel is beyond the grid: with an even row pitch the second slot
// of a pair that starts inside a row is inside the row too (in the padding
// when the second voxel is beyond the grid, where the kernel computes zero
// labels and flows; the tensor maps end at the grid, so nothing reads it).
template <typename T> __device__ __forceinline__ void st_pair_u_padded(T* p, float2 v) {
    if constexpr (std::is_same<T, __half>::value) v = make_float2(fmaxf(v.x, F16_U_FLOOR), fmaxf(v.y, F16_U_FLOOR));
    stv2<T>(p, v);
}

// Synchronisation.  No block barrier holds the warps in step.  Staged plane
// s of the chunk (plane z0-1 + s; s = 0 holds only the flows of plane z0-1)
// sits in stage s % 4 and is handed over by that stage's TMA barrier; its
// prox writes g plane (s-1) % 4, and every thread then arrives on that g
// plane's barrier (its g values are written, its reads of stage s are done)
// and waits on the barrier of plane s-1 just before the flow step that reads
// g of plane s-1 at the neighbours.  A warp may therefore run up to one plane
// ahead of the slowest one, and the warps' phases interleave.  The rings are
// deep enough: the TMA load of plane s+3, issued in plane s right after the
// wait on plane s-1's g barrier, refills the stage of plane s-1, whose readers
// have all arrived on that barrier (planes s+1 and s+2 are in flight, so a
// load is requested two and a half planes ahead of its use; planes 0-2 are
// requested before the loop, 3-4 at the start of plane 1); the prox of plane s overwrites the g plane of plane
// s-4, whose last readers (the flow steps in plane s-3) arrived on the
// barrier of plane s-2 after them, which the writing thread has passed.  A
// barrier's k-th use (k = 0, 1, ...) is waited on with parity k & 1: stage b
// is used at s = b + 4k, g plane b by the prox of s = b + 1 + 4k.  The plane
// loop is unrolled twice, so that the values carried from one plane to the
// next (g, flows, field) alternate between two register sets instead of
// being copied.
//
// EXACT: the problem has exactly MAXL labels (no per-label guards).
// WITH_E: also reduce E(u) and P(q) of the input state into one (E, P)
// partial per CTA, as fused_tma_kernel does (P of plane p from the prox's
// per-voxel minimum, E of plane p-1 in the flow phase, whose z-difference
// takes plane p's staged u); the update itself is the same arithmetic.
template <int MAXL, typename T, bool EXACT, bool WITH_E, bool IDX32>
__global__ void __launch_bounds__(X2_NT, 1)
fused_tma_x2_kernel(const StepArgs<MAXL, MAXL> a, const __grid_constant__ TmaMaps maps, double* partial) {
    static_assert(MAXL % 4 == 0, "labels are split in four");
    constexpr int DIM = 3;
    constexpr int QL = MAXL / 4;
    using Lay = X2Layout<MAXL, T>;
    constexpr int NS = Lay::STAGES;
    constexpr int NG = Lay::GBUF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ double sE[X2_NT / 32], sP[X2_NT / 32];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x;
    const int h = t & 3;
    const int v = t >> 2;
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
    const unsigned bar0 = smem_addr(smem + Lay::bar_off);  // stage barriers
    const unsigned gbar0 = bar0 + 8 * NS;                   // g plane barriers
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
        for (int k = 0; k < NS; ++k) mbar_init(bar0 + 8 * k, 1);
        for (int k = 0; k < NG; ++k) mbar_init(gbar0 + 8 * k, X2_NT);
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

    // pair of this thread quad: owned pairs first (v < 128), then the y-halo
    // row (ey = 8), then the x-halo column (ex = 32)
    constexpr int OWNED = (FTX / 2) * FTY;
    const bool inE = v < X2_PAIRS;
    const int ex = v < OWNED ? 2 * (v & (FTX / 2 - 1)) : v < OWNED + FTX / 2 ? 2 * (v - OWNED) : FTX;
    const int ey = v < OWNED ? v / (FTX / 2) : v < OWNED + FTX / 2 ? FTY : v - (OWNED + FTX / 2);
    const int xe = x0 + ex, ye = y0 + ey;
    const bool validE = inE && xe < a.nx && ye < a.ny;
    const bool both = validE && xe + 1 < a.nx;  // second voxel inside the grid
    const bool ownerE = validE && v < OWNED;
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * Lay::QBX + (ex + Lay::QOFF);
    const long long vox = (long long)ye * a.px + xe;
    // minus the step c tau, zero at the last index of each axis
    const float2 ncx = make_float2(xe < a.nx - 1 ? -a.ctau : 0.f, xe + 1 < a.nx - 1 ? -a.ctau : 0.f);
    const float cyv = ye < a.ny - 1 ? -a.ctau : 0.f;
    const float2 ncy = make_float2(cyv, cyv);

    for (int k = t; k < NG * Lay::g_elems; k += X2_NT) gbuf[k] = 0.f;
    float cap[QL];
#pragma unroll
    for (int i = 0; i < QL; ++i) cap[i] = (EXACT || h + 4 * i < nl) ? a.s_node[h + 4 * i] : 0.f;
    float2 gprev[QL], gcur[QL], qxp[QL], qyp[QL], qzp[QL];
    float2 sprev = make_float2(1.f, 1.f);
    const float2 zero2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < QL; ++i) gprev[i] = gcur[i] = qxp[i] = qyp[i] = qzp[i] = zero2;
    bool ok = mbar_wait_bounded(bar0, 0u);
    if (ok && validE) {
        const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + Lay::q_off);
#pragma unroll
        for (int i = 0; i < QL; ++i) {
            const int j = h + 4 * i;
            if (EXACT || j < nl) qzp[i] = lds2<T>(q0 + (j * DIM + 2) * qstride + qi);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the zeroed g planes and the reads of stage 0 are complete everywhere
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        s_abort = 1;
    }
    // WITH_E: this pair's staged u and the x / y part of its input gradient
    // norm, carried to the next plane, which supplies the z difference
    float2 uin_prev[QL], txy_prev[QL];
#pragma unroll
    for (int i = 0; i < QL; ++i) uin_prev[i] = txy_prev[i] = zero2;
    SumF sumE, sumP;
    bool bad = false;
    int p_stop = z0 - 1;
#pragma unroll 2
    for (int p = z0; p <= z1 && !s_abort; ++p) {
        const int s = p - z0 + 1;
        const int cs = s % NS;
        if (s == 1 && t == 0) {
            for (int k = 2; k <= 3; ++k)
                if (p + k <= z1 && p + k < a.nz) {
                    issue(p + k, (s + k) % NS, false);
                    inflight_hi = p + k;
                }
        }
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + ((s + NG - 1) % NG) * Lay::g_elems;        // plane s
        const float* gP = gbuf + ((s + NG - 2) % NG) * Lay::g_elems;  // plane s-1
        if (p < a.nz && !mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / NS) & 1))) {
            atomicOr(a.flags, FLAG_TIMEOUT);
            s_abort = 1;
            break;
        }
        float2 qxc[QL], qyc[QL], qzc[QL], uin[QL], txy[QL];
#pragma unroll
        for (int i = 0; i < QL; ++i) qxc[i] = qyc[i] = qzc[i] = uin[i] = txy[i] = zero2;
        float2 scur = make_float2(1.f, 1.f);
        float eD = 0.f;  // sum of D u over this thread's labels of plane p (WITH_E)

        // ---- label prox of plane p on the halo-extended tile
        if (p < a.nz) {
            const T* uS = reinterpret_cast<const T*>(cst + Lay::u_off);
            const float* dS = reinterpret_cast<const float*>(cst + Lay::d_off);
            const T* qS = reinterpret_cast<const T*>(cst + Lay::q_off);
            if (has_S && ownerE) scur = *reinterpret_cast<const float2*>(cst + Lay::s_off + 4 * (ey * FTX + ex));
            // divergence without boundary tests (the last-index normal flow
            // is an invariant zero; the box is zero-filled outside the grid)
            float2 u[QL], d[QL];
            float2 mloc = make_float2(3.0e38f, 3.0e38f);
#pragma unroll
            for (int i = 0; i < QL; ++i) {
                const int j = h + 4 * i;
                u[i] = d[i] = zero2;
                if (validE && (EXACT || j < nl)) {
                    u[i] = lds2<T>(uS + j * ustride + ui);
                    const T* qx = qS + (j * DIM + 0) * qstride + qi;
                    const T* qy = qS + (j * DIM + 1) * qstride + qi;
                    qxc[i] = lds2<T>(qx);
                    qyc[i] = lds2<T>(qy);
                    qzc[i] = lds2<T>(qS + (j * DIM + 2) * qstride + qi);
                    const float2 qxl = make_float2(lds<T>(qx - 1), qxc[i].x);  // q_x at x-1, x
                    const float2 qyl = lds2<T>(qy - Lay::QBX);
                    const float2 dv = f2add(f2add(f2sub(qxc[i], qxl), f2sub(qyc[i], qyl)), f2sub(qzc[i], qzp[i]));
                    const float2 Dv = *reinterpret_cast<const float2*>(dS + j * ustride + ui);
                    d[i] = f2add(Dv, dv);
                    mloc.x = fminf(mloc.x, d[i].x);
                    mloc.y = fminf(mloc.y, d[i].y);
                    if constexpr (WITH_E) {
                        uin[i] = u[i];
                        if (ownerE) {
                            const T* uj = uS + j * ustride + ui;
                            // forward differences, zero at the last index
                            const float2 ux1 = make_float2(u[i].y, lds<T>(uj + 2));
                            const float2 uy1 = lds2<T>(uj + TMA_BX);
                            const float2 gx = f2sub(ux1, u[i]), gy = f2sub(uy1, u[i]);
                            const float gxa = ncx.x != 0.f ? gx.x : 0.f, gxb = ncx.y != 0.f ? gx.y : 0.f;
                            const float gya = ncy.x != 0.f ? gy.x : 0.f, gyb = ncy.y != 0.f ? gy.y : 0.f;
                            txy[i] = a.aniso ? make_float2(fabsf(gxa) + fabsf(gya), fabsf(gxb) + fabsf(gyb))
                                             : make_float2(fmaf(gxa, gxa, gya * gya), fmaf(gxb, gxb, gyb * gyb));
                            if (p < z1) eD = fmaf(Dv.x, u[i].x, both ? fmaf(Dv.y, u[i].y, eD) : eD);
                        }
                    }
                }
            }
            float2 m;
            m.x = fminf(mloc.x, __shfl_xor_sync(0xffffffffu, mloc.x, 1));
            m.y = fminf(mloc.y, __shfl_xor_sync(0xffffffffu, mloc.y, 1));
            m.x = fminf(m.x, __shfl_xor_sync(0xffffffffu, m.x, 2));
            m.y = fminf(m.y, __shfl_xor_sync(0xffffffffu, m.y, 2));
            // the per-voxel minimum is the dual term of the voxel
            if constexpr (WITH_E) {
                if (ownerE && p < z1 && h == 0) {
                    sumP.add(m.x);
                    if (both) sumP.add(m.y);
                }
            }
            if (a.literal) m = zero2;
            // 2^((d - m) kexp) = 2^(d kexp - m kexp)
            const float2 k2 = make_float2(kexp, kexp);
            const float2 mk = make_float2(-m.x * kexp, -m.y * kexp);
            float2 sloc = zero2;
#pragma unroll
            for (int i = 0; i < QL; ++i) {
                const int j = h + 4 * i;
                if (validE && (EXACT || j < nl)) {
                    const float2 ea = f2fma(d[i], k2, mk);
                    u[i] = f2mul(u[i], make_float2(ex2_approx(ea.x), ex2_approx(ea.y)));
                    sloc = f2add(sloc, u[i]);
                }
            }
            float2 sum;
            sum.x = sloc.x + __shfl_xor_sync(0xffffffffu, sloc.x, 1);
            sum.y = sloc.y + __shfl_xor_sync(0xffffffffu, sloc.y, 1);
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, 2);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, 2);
            if (validE) {
                if (!((sum.x > 0.f) && (sum.x <= 3.0e38f))) bad = true;
                if (both && !((sum.y > 0.f) && (sum.y <= 3.0e38f))) bad = true;
                // a second voxel beyond the grid is zero (its staged u is zero)
                const float2 inv = make_float2(rcp_fast(sum.x), both ? rcp_fast(sum.y) : 0.f);
#pragma unroll
                for (int i = 0; i < QL; ++i) {
                    const int j = h + 4 * i;
                    if (EXACT || j < nl) {
                        const float2 un = f2mul(u[i], inv);
                        gcur[i] = a.literal ? make_float2(u[i].x, both ? u[i].y : 0.f) : un;
                        *reinterpret_cast<float2*>(gC + j * ustride + ui) = gcur[i];
                        if (ownerE && p < z1) st_pair_u_padded<T>(slot_ptr<IDX32>(uout, j, p, n, plane, vox), un);
                    }
                }
            }
        }

        // g of plane p written, stage of plane p read (before a later TMA
        // load refills it)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(gbar0 + 8 * ((s + NG - 1) % NG));

        // ---- flow step of plane p-1 at the owned pair: g of plane p-1 at
        // x+2 and y+1 from shared memory (once every thread has written it),
        // own g of planes p-1 and p from registers
        const int pm = p - 1;
        if (pm >= z0 && !mbar_wait_bounded(gbar0 + 8 * ((s + NG - 2) % NG), (unsigned)(((s - 2) / NG) & 1))) {
            atomicOr(a.flags, FLAG_TIMEOUT);
            s_abort = 1;
            break;
        }
        if (pm >= z0 && t == 0 && p + 3 <= z1 && p + 3 < a.nz) {
            issue(p + 3, (s + 3) % NS, false);
            inflight_hi = p + 3;
        }
        if (pm >= z0 && ownerE) {
            const float czv = pm < a.nz - 1 ? -a.ctau : 0.f;
            const float2 ncz = make_float2(czv, czv);
            float eloc = 0.f;
#pragma unroll
            for (int i = 0; i < QL; ++i) {
                const int j = h + 4 * i;
                if (EXACT || j < nl) {
                    const float* gj = gP + j * ustride + ui;
                    const float2 g0 = gprev[i];
                    const float2 gx1 = make_float2(g0.y, gj[2]);                   // g at x+1, x+2
                    const float2 gy1 = *reinterpret_cast<const float2*>(gj + TMA_BX);  // g at y+1
                    // y = q - c tau grad g
                    float2 yx = f2fma(ncx, f2sub(gx1, g0), qxp[i]);
                    float2 yy = f2fma(ncy, f2sub(gy1, g0), qyp[i]);
                    float2 yz = f2fma(ncz, f2sub(gcur[i], g0), qzp[i]);
                    const float2 sj = f2mul(make_float2(cap[i], cap[i]), sprev);
                    if constexpr (WITH_E) {
                        // TV term of plane p-1 on the input labelling
                        const float2 gz = czv != 0.f ? f2sub(uin[i], uin_prev[i]) : zero2;
                        const float2 tp = txy_prev[i];
                        const float na = a.aniso ? tp.x + fabsf(gz.x) : sqrt_approx(fmaf(gz.x, gz.x, tp.x));
                        const float nb = a.aniso ? tp.y + fabsf(gz.y) : sqrt_approx(fmaf(gz.y, gz.y, tp.y));
                        eloc = fmaf(sj.x, na, eloc);
                        if (both) eloc = fmaf(sj.y, nb, eloc);
                    }
                    float2 f;
                    if (a.aniso) {
                        yx = make_float2(fminf(fmaxf(yx.x, -sj.x), sj.x), fminf(fmaxf(yx.y, -sj.y), sj.y));
                        yy = make_float2(fminf(fmaxf(yy.x, -sj.x), sj.x), fminf(fmaxf(yy.y, -sj.y), sj.y));
                        yz = make_float2(fminf(fmaxf(yz.x, -sj.x), sj.x), fminf(fmaxf(yz.y, -sj.y), sj.y));
                    } else {
                        const float2 r2 = f2fma(yz, yz, f2fma(yy, yy, f2mul(yx, yx)));
                        f.x = sj.x > 0.f ? fminf(1.0f, sj.x * rsqrt_approx(r2.x)) : 0.f;
                        f.y = sj.y > 0.f ? fminf(1.0f, sj.y * rsqrt_approx(r2.y)) : 0.f;
                        yx = f2mul(yx, f);
                        yy = f2mul(yy, f);
                        yz = f2mul(yz, f);
                    }
                    stv2<T>(slot_ptr<IDX32>(qout, j * DIM + 0, pm, n, plane, vox), yx);
                    stv2<T>(slot_ptr<IDX32>(qout, j * DIM + 1, pm, n, plane, vox), yy);
                    stv2<T>(slot_ptr<IDX32>(qout, j * DIM + 2, pm, n, plane, vox), yz);
                }
            }
            if constexpr (WITH_E) sumE.add(eloc);
        }
        if constexpr (WITH_E) sumE.add(eD);
#pragma unroll
        for (int i = 0; i < QL; ++i) {
            gprev[i] = gcur[i];
            qxp[i] = qxc[i];
            qyp[i] = qyc[i];
            qzp[i] = qzc[i];
            uin_prev[i] = uin[i];
            txy_prev[i] = txy[i];
        }
        sprev = scur;
        p_stop = p;
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    // after an abort, the copies still in flight land before the block exits
    if (t == 0) {
        for (int p = p_stop + 1; p <= inflight_hi; ++p) {
            const int s = p - z0 + 1;
            mbar_wait_bounded(bar0 + 8 * (s % NS), (unsigned)((s / NS) & 1));
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
            for (int k = 0; k < X2_NT / 32; ++k) {
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
