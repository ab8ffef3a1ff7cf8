// pfm_tma_dag4.cuh -- TMA-pipelined fused iteration for label DAGs with at
// most four non-end-label nodes (Algorithm 2 in its path-weight form).
//
// Every end-label j has its own node (path weight W_(j,j) = 1) and is reached
// from the source through the other nodes A ("inner" nodes) with path weights
// W_(A,j).  By the definition of the flow excess (Section 3.3) and the
// bottom-up accumulation of Algorithm 2,
//   d_j = D_j + e_j + sum_A W_(A,j) e_A,   e = div q,
//   g_A = sum_j W_(A,j) g_j,
// whatever the DAG's depth.  With at most four inner nodes both sums are a
// fixed handful of register operations: the DAGMF workload (four inner nodes,
// end-labels with one or two parents) and the HMF trees qualify.
//
// Layout of the work: the general DAG kernel's plane pipeline (32 x 4 tiles,
// three-stage cp.async.bulk.tensor ring, two planes in flight, one barrier
// per plane, flows / g / S of the voxel carried in registers) with four
// threads per voxel.  Lane h of a voxel takes end-labels j = h, h + 4,
// h + 8 (slot s holds j = 4 s + h) and inner node h.  Per plane:
//   prox: lane h forms the divergence of its end-labels' flows and of inner
//         node h's flow; the four inner divergences reach every lane by
//         shuffles; d_j, the per-voxel minimum (two xor shuffles), the
//         shifted exponential, the normaliser (two xor shuffles); each lane
//         forms its end-labels' contributions W_(A,j) g_j to the four inner
//         nodes, and a reduce-scatter over the four lanes (three shuffles)
//         leaves g_A with lane A;
//   flow: lane h steps the flows of its end-labels and of inner node h.
// The tile body is a device function shared by the single-problem kernel and
// the batched persistent kernel (which draws (member, tile, z-chunk) items
// from a counter, like the general batched DAG kernel).
#pragma once

#include "pfm_tma_tree.cuh"

namespace pfm {

constexpr int DAG4_INNER = 4;                    // inner nodes (one per lane)
constexpr int DAG4_SLOTS = 3;                    // end-labels per lane
constexpr int DAG4_MAXL = 4 * DAG4_SLOTS;        // 12 end-labels

// Shape of such a DAG: inner node ids (-1: unused lane), the own node of
// every end-label, and the path weights W_(inner k, end-label j).
struct Dag4Shape {
    int ni;                              // inner nodes
    int inner[DAG4_INNER];
    int lnode[DAG4_MAXL];
    float w[DAG4_MAXL][DAG4_INNER];
};

// One tile (bx, by) of z-chunk bz of one problem; the layout (box width,
// offsets) is the tree kernel's for (nl, nn).  Returns false after a
// timed-out wait (FLAG_TIMEOUT raised; the caller drains the ring and stops).
// Every thread of the CTA calls it; it ends with a CTA barrier.
template <int DIM, typename T, bool IDX32>
__device__ __forceinline__ bool dag4_tma_tile(const StepArgs<DMAX, DMAX>& a, const TmaMaps& maps,
                                              const Dag4Shape& sh, int bx, int by, int bz, unsigned char* smem,
                                              unsigned bar0, DagRing& ring) {
    constexpr int QOFF = 16 / (int)sizeof(T);
    constexpr int ustride = DAG_UY * TMA_BX;
    constexpr int NS = DAG4_SLOTS;
    constexpr int NI = DAG4_INNER;
    const int nl = a.nl, nn = a.nn;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px, literal = a.literal, aniso = a.aniso;
    const float ctau = a.ctau;
    const TreeTmaLayout lay(nl, nn, DIM, (int)sizeof(T));
    const int QBX = lay.qbx;
    const int qstride = DAG_QY * QBX;
    const int t = threadIdx.x;
    const int h = t & 3;
    const int v = t >> 2;
    const int x0 = bx * FTX, y0 = by * DTY;
    const int z0 = bz * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const long long n = a.n;
    const long long plane = (long long)px * ny;
    T* __restrict__ uout = static_cast<T*>(a.u_out);
    T* __restrict__ qout = static_cast<T*>(a.q_out);
    const int has_S = a.S != nullptr;
    const unsigned bytes_u = (unsigned)(nl * ustride * sizeof(T));
    const unsigned bytes_d = (unsigned)(nl * ustride * 4);
    const unsigned bytes_q = (unsigned)(DIM * nn * qstride * sizeof(T));
    const unsigned bytes_s = has_S ? (unsigned)(FTX * DTY * 4) : 0u;
    const float kexp = -a.inv_c * 1.4426950408889634f;  // exp(-(d-m)/c) = 2^((d-m) kexp)
    float* gbuf = reinterpret_cast<float*>(smem + lay.g_off);
    const int g_elems = nn * ustride;

    auto stage_ptr = [&](int k) { return smem + k * lay.stage_bytes; };
    auto issue = [&](int p, int k, bool flows_only) {
        const unsigned bar = bar0 + 8 * k;
        ring.pending |= 1u << k;
        unsigned char* st = stage_ptr(k);
        mbar_expect_tx(bar, flows_only ? bytes_q : bytes_u + bytes_d + bytes_q + bytes_s);
        tma_load_4d(smem_addr(st + lay.q_off), &maps.q, x0 - QOFF, y0 - 1, p, 0, bar);
        if (!flows_only) {
            tma_load_4d(smem_addr(st + lay.u_off), &maps.u, x0, y0, p, 0, bar);
            tma_load_4d(smem_addr(st + lay.d_off), &maps.D, x0, y0, p, 0, bar);
            if (has_S) tma_load_3d(smem_addr(st + lay.s_off), &maps.S, x0, y0, p, bar);
        }
    };
    // plane p of the chunk lives in stage (p - z0 + 1) % 3; the ring runs two
    // planes ahead
    auto wait_stage = [&](int k) {
        const bool r = mbar_wait_bounded(bar0 + 8 * k, (ring.phase >> k) & 1u);
        if (r) {
            ring.phase ^= 1u << k;
            if (t == 0) ring.pending &= ~(1u << k);
        }
        return r;
    };
    if (t == 0) {
        issue(z0 - 1, 0, true);
        issue(z0, 1, false);
        if (z0 + 1 <= z1 && z0 + 1 < nz) issue(z0 + 1, 2, false);
    }

    // voxel of this thread quad on the halo-extended 33 x 5 tile (owned
    // first, then the y-halo row, then the x-halo column)
    const bool inE = v < DNE;
    const int ex = v < FTX * DTY ? (v & (FTX - 1)) : v < FTX * DTY + FTX ? v - FTX * DTY : FTX;
    const int ey = v < FTX * DTY ? v / FTX : v < FTX * DTY + FTX ? DTY : v - (FTX * DTY + FTX);
    const int xe = x0 + ex, ye = y0 + ey;
    const bool validE = inE && xe < nx && ye < ny;
    const bool ownerE = validE && v < FTX * DTY;
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * QBX + (ex + QOFF);
    const long long vox = (long long)ye * px + xe;
    const float cx = xe < nx - 1 ? ctau : 0.f;
    const float cy = ye < ny - 1 ? ctau : 0.f;
    const int lane0 = (t & 31) & ~3;  // first lane of this voxel's quad

    for (int k = t; k < 2 * g_elems; k += DAG_TMA_NT) gbuf[k] = 0.f;
    // this lane's end-labels (slot s: j = 4 s + h; lnd < 0: none) and inner
    // node, read once
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
    auto uo = [&](int s) { return (4 * s + h) * ustride + ui; };
    auto qo = [&](int s) { return lnd[s] * (DIM * qstride) + qi; };
    auto go = [&](int s) { return lnd[s] * ustride + ui; };
    const int qo_i = (inn >= 0 ? inn : 0) * (DIM * qstride) + qi;
    const int go_i = (inn >= 0 ? inn : 0) * ustride + ui;
    float gprev[NS], gcur[NS], qxp[NS], qyp[NS], qzp[NS];
    float gprev_i = 0.f, gcur_i = 0.f, qxp_i = 0.f, qyp_i = 0.f, qzp_i = 0.f;
    float sprev = 1.0f;
#pragma unroll
    for (int s = 0; s < NS; ++s) gprev[s] = gcur[s] = qxp[s] = qyp[s] = qzp[s] = 0.f;
    // z flows of plane z0-1 (its x / y flow steps belong to the previous chunk)
    bool ok = wait_stage(0);
    if constexpr (DIM == 3) {
        if (ok && validE) {
            const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + lay.q_off);
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (lnd[s] >= 0) qzp[s] = lds<T>(q0 + qo(s) + 2 * qstride);
            if (inn >= 0) qzp_i = lds<T>(q0 + qo_i + 2 * qstride);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        return false;
    }
    bool bad = false;
    bool alive = true;
    for (int p = z0; p <= z1; ++p) {
        const int s_ = p - z0 + 1;
        const int cs = s_ % 3, ps = (s_ + 2) % 3;
        // stage ps held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 <= z1 && p + 2 < nz) issue(p + 2, ps, false);
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + (p & 1) * g_elems;
        const float* gP = gbuf + ((p + 1) & 1) * g_elems;
        ok = true;
        if (p < nz) ok = wait_stage(cs);
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        float qxc[NS], qyc[NS], qzc[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) qxc[s] = qyc[s] = qzc[s] = 0.f;
        float qxc_i = 0.f, qyc_i = 0.f, qzc_i = 0.f;
        float scur = 1.0f;

        // ---- label prox of plane p on the halo-extended tile (uniform branch)
        if (p < nz) {
            const T* uS = reinterpret_cast<const T*>(cst + lay.u_off);
            const float* dS = reinterpret_cast<const float*>(cst + lay.d_off);
            const T* qS = reinterpret_cast<const T*>(cst + lay.q_off);
            if (has_S && ownerE) scur = reinterpret_cast<const float*>(cst + lay.s_off)[ey * FTX + ex];
            // divergence (no boundary tests: the last-index normal flow is an
            // invariant zero, the box is zero-filled outside the grid)
            auto divergence = [&](int qoff, float& qx, float& qy, float& qz, float qzprev) {
                const T* bxp = qS + qoff;
                const T* byp = bxp + qstride;
                qx = lds<T>(bxp);
                qy = lds<T>(byp);
                float dv = (qx - lds<T>(bxp - 1)) + (qy - lds<T>(byp - QBX));
                if constexpr (DIM == 3) {
                    qz = lds<T>(bxp + 2 * qstride);
                    dv += qz - qzprev;
                }
                return dv;
            };
            float ei = 0.f;  // divergence of this lane's inner node
            if (validE && inn >= 0) ei = divergence(qo_i, qxc_i, qyc_i, qzc_i, qzp_i);
            float ep[NI];    // every inner node's divergence at this voxel
#pragma unroll
            for (int k = 0; k < NI; ++k) ep[k] = __shfl_sync(0xffffffffu, ei, lane0 + k);
            float u[NS], d[NS];
            float mloc = 3.0e38f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                u[s] = 0.f;
                d[s] = 0.f;
                if (validE && lnd[s] >= 0) {
                    u[s] = lds<T>(uS + uo(s));
                    float dj = dS[uo(s)] + divergence(qo(s), qxc[s], qyc[s], qzc[s], qzp[s]);
#pragma unroll
                    for (int k = 0; k < NI; ++k) dj = fmaf(wv[s][k], ep[k], dj);
                    d[s] = dj;
                    mloc = fminf(mloc, dj);
                }
            }
            float m = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
            m = fminf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            if (literal) m = 0.f;
            float sloc = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (validE && lnd[s] >= 0) {
                    u[s] *= ex2_approx((d[s] - m) * kexp);
                    sloc += u[s];
                }
            }
            float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            if (validE && !((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
            const float inv = rcp_fast(sum);
            // end-labels' g (normalised, or unnormalised as printed), stored
            // labelling, and this lane's contributions W_(A,j) g_j to each
            // inner node A
            float part[NI];
#pragma unroll
            for (int k = 0; k < NI; ++k) part[k] = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (validE && lnd[s] >= 0) {
                    const float un = u[s] * inv;
                    const float gk = literal ? u[s] : un;
                    gcur[s] = gk;
                    gC[go(s)] = gk;
                    if (ownerE && p < z1) stu<T>(slot_ptr<IDX32>(uout, 4 * s + h, p, n, plane, vox), un);
#pragma unroll
                    for (int k = 0; k < NI; ++k) part[k] = fmaf(wv[s][k], gk, part[k]);
                }
            }
            // reduce-scatter over the quad: lane h ends with the sum of part[h]
            // (the first shuffle step pairs lanes two apart, the second neighbours)
            const bool hi2 = (h & 2) != 0, hi1 = (h & 1) != 0;
            const float s0 = hi2 ? part[0] : part[2], s1 = hi2 ? part[1] : part[3];
            const float k0 = hi2 ? part[2] : part[0], k1 = hi2 ? part[3] : part[1];
            const float r0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 2);
            const float r1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 2);
            gcur_i = (hi1 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, hi1 ? r0 : r1, 1);
            if (validE && inn >= 0) gC[go_i] = gcur_i;
        }

        // ---- flow step of plane p-1 at the owned voxel: neighbours' g of
        // plane p-1 from shared memory (visible since the last barrier), own
        // g of planes p-1 and p from registers
        const int pm = p - 1;
        if (pm >= z0 && ownerE) {
            const float sf = sprev;
            const float cz = pm < nz - 1 ? ctau : 0.f;
            auto flow_step = [&](int node, int goff, float g0, float g1, float qx, float qy, float qz, float capn) {
                const float* gA = gP + goff;
                float yv[DIM];
                yv[0] = qx - cx * (gA[1] - g0);
                yv[1] = qy - cy * (gA[TMA_BX] - g0);
                if constexpr (DIM == 3) yv[2] = qz - cz * (g1 - g0);
                project_nb<DIM>(yv, capn * sf, aniso);
#pragma unroll
                for (int c = 0; c < DIM; ++c) stv<T>(slot_ptr<IDX32>(qout, node * DIM + c, pm, n, plane, vox), yv[c]);
            };
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (lnd[s] >= 0) flow_step(lnd[s], go(s), gprev[s], gcur[s], qxp[s], qyp[s], qzp[s], capl[s]);
            if (inn >= 0) flow_step(inn, go_i, gprev_i, gcur_i, qxp_i, qyp_i, qzp_i, capi);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            gprev[s] = gcur[s];
            qxp[s] = qxc[s];
            qyp[s] = qyc[s];
            qzp[s] = qzc[s];
        }
        gprev_i = gcur_i;
        qxp_i = qxc_i;
        qyp_i = qyc_i;
        qzp_i = qzc_i;
        sprev = scur;
        // order this plane's shared-memory accesses before the TMA that
        // refills a stage; one barrier per plane, which also carries a
        // timed-out wait of any thread to the whole CTA
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            alive = false;
            break;
        }
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    return alive;
}

// One problem: CTA = (x tile, y tile, z chunk).
template <int DIM, typename T, bool IDX32>
__global__ void __launch_bounds__(DAG_TMA_NT, 1)
dag4_tma_kernel(const StepArgs<DMAX, DMAX> a, const __grid_constant__ TmaMaps maps,
                const __grid_constant__ Dag4Shape shape) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = dag_smem_base(smem_raw);
    const TreeTmaLayout lay(a.nl, a.nn, DIM, (int)sizeof(T));
    const unsigned bar0 = smem_addr(smem + lay.bar_off);
    if (threadIdx.x == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    DagRing ring;
    if (!dag4_tma_tile<DIM, T, IDX32>(a, maps, shape, blockIdx.x, blockIdx.y, blockIdx.z, smem, bar0, ring) &&
        threadIdx.x == 0)
        dag_ring_drain(bar0, ring);
}

// Many problems in one persistent launch: CTAs take (problem, x tile, y tile,
// z chunk) items in list order from a global counter (zeroed before the
// launch); args, maps and shapes are per problem (this launch's parity).
// The mbarrier ring carries over from item to item; dynamic shared memory is
// sized for the largest member layout, the barriers past all of them.
template <int DIM, typename T, bool IDX32>
__global__ void __launch_bounds__(DAG_TMA_NT, 1)
batched_dag4_tma_kernel(const StepArgs<DMAX, DMAX>* __restrict__ args, const TmaMaps* __restrict__ maps,
                        const Dag4Shape* __restrict__ shapes, const int4* __restrict__ items, int n_items,
                        int bar_off, int* next_item) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    unsigned char* smem = dag_smem_base(smem_raw);
    const unsigned bar0 = smem_addr(smem + bar_off);
    if (threadIdx.x == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    DagRing ring;
    bool alive = true;
    while (alive) {
        // the previous item ended with a CTA barrier: s_item and the stages are free
        if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        alive = dag4_tma_tile<DIM, T, IDX32>(args[w.x], maps[w.x], shapes[w.x], w.y, w.z, w.w, smem, bar0, ring);
    }
    if (!alive && threadIdx.x == 0) dag_ring_drain(bar0, ring);
}

}  // namespace pfm
