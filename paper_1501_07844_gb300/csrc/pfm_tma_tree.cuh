// pfm_tma_tree.cuh -- TMA-pipelined fused iteration for two-level label
// trees (the hierarchical model HMF of Section 3.4 with source S -> inner
// nodes -> end-labels; Algorithm 2 on a tree).
//
// On such a tree the orders O / O^-1 of Algorithm 2 are one step each: an
// end-label's excess is its own divergence plus its parent's,
//   d_j = D_j + e_j + w_(A,j) e_A,   e = div q,
// and the bottom-up accumulation of an inner node is the weighted sum of its
// end-labels,  g_A = sum_j w_(A,j) g_j.  The general DAG kernel walks
// runtime path-weight lists for both; here the tree shape is fixed at
// creation and the sums are a handful of register operations and lane
// shuffles.
//
// Layout of the work: the general DAG kernel's plane pipeline (32 x 4 tiles,
// three-stage cp.async.bulk.tensor ring, two planes in flight, one barrier
// per plane, flows / g / S of the voxel carried in registers) with four
// threads per voxel.  The end-labels form groups (group k = the children of
// inner node k, at most four each); lane h of a voxel takes end-label h of
// every group and, for h < #groups, inner node h.  Per plane:
//   prox: lane h forms the divergence of its end-labels' flows and of inner
//         node h's flow; the inner divergences reach the other lanes by
//         shuffles; d, the per-voxel minimum (two xor shuffles), the shifted
//         exponential, the normaliser (two xor shuffles); g_A of every group
//         by an xor-butterfly sum over the four lanes;
//   flow: lane h steps the flows of its end-labels and of inner node h.
#pragma once

#include "pfm_tma_dag.cuh"

namespace pfm {

constexpr int TREE_MAXG = 4;   // groups (inner nodes)
constexpr int TREE_FAN = 4;    // end-labels per group = lanes per voxel

// Shape of a two-level tree.  Group k: inner node inner[k] (-1: the group's
// end-labels hang directly under S and have no common parent flow), its
// end-labels h < n[k]: leaf index leaf[k][h] (into u and D), node id
// lnode[k][h] (into q and the capacities), weight w[k][h] = w_(inner,leaf).
struct TreeShape {
    int ng;
    int n[TREE_MAXG];
    int inner[TREE_MAXG];
    int leaf[TREE_MAXG][TREE_FAN];
    int lnode[TREE_MAXG][TREE_FAN];
    float w[TREE_MAXG][TREE_FAN];
};

// Shared-memory layout: per stage u, D (n_leaf), the flows of all nn nodes
// and S; two planes of g for every node.  The flow box is one box of
// qbx x 6 rows per node component; the four lanes of a voxel read four
// different nodes at the same position, so the node stride (3 * 6 * qbx
// elements) should not be a multiple of 16 banks: the box is widened on the
// right (qbx 44 for FP32, 56 for 16-bit types: a node stride of 24 banks
// mod 32) when three stages still fit, else it keeps the 32 + 2 * 16 bytes
// the halo needs (qbx 40 / 48: two lanes of a quad share a bank).
struct TreeTmaLayout {
    int qbx, u_off, d_off, q_off, s_off, stage_bytes, g_off, bar_off, total;
    __host__ __device__ static int a128(int b) { return (b + 127) / 128 * 128; }
    __host__ __device__ TreeTmaLayout(int nl, int nn, int dim, int es) {
        qbx = es == 4 ? 44 : 56;
        set(nl, nn, dim, es);
        if (total + 64 > 227 * 1024) {
            qbx = FTX + 2 * (16 / es);
            set(nl, nn, dim, es);
        }
    }
    __host__ __device__ void set(int nl, int nn, int dim, int es) {
        u_off = 0;
        d_off = a128(nl * DAG_UY * TMA_BX * es);
        q_off = d_off + a128(nl * DAG_UY * TMA_BX * 4);
        s_off = q_off + a128(dim * nn * DAG_QY * qbx * es);
        stage_bytes = s_off + a128(FTX * DTY * 4);
        g_off = TMA_STAGES * stage_bytes;
        bar_off = g_off + a128(2 * nn * DAG_UY * TMA_BX * 4);
        total = bar_off + 64 + 128;
    }
};

// G: groups the kernel is compiled for (>= tree.ng; 3 or 4): the per-group
// state lives in registers, so a tree of three groups runs the G = 3 form.
template <int DIM, typename T, bool IDX32, int G>
__global__ void __launch_bounds__(DAG_TMA_NT, 1)
tree_tma_kernel(const StepArgs<DMAX, DMAX> a, const __grid_constant__ TmaMaps maps,
                const __grid_constant__ TreeShape tree) {
    static_assert(G >= 1 && G <= TREE_MAXG, "group count");
    constexpr int QOFF = 16 / (int)sizeof(T);
    constexpr int ustride = DAG_UY * TMA_BX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    unsigned char* smem = dag_smem_base(smem_raw);
    const int nl = a.nl, nn = a.nn, ng = tree.ng;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px, literal = a.literal, aniso = a.aniso;
    const float ctau = a.ctau;
    const TreeTmaLayout lay(nl, nn, DIM, (int)sizeof(T));
    const int QBX = lay.qbx;             // flow box width (elements)
    const int qstride = DAG_QY * QBX;    // one flow component of one node
    const int t = threadIdx.x;
    const int h = t & 3;
    const int v = t >> 2;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * DTY;
    const int z0 = blockIdx.z * a.zc;
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
    const unsigned bar0 = smem_addr(smem + lay.bar_off);

    auto stage_ptr = [&](int k) { return smem + k * lay.stage_bytes; };
    auto issue = [&](int p, int k, bool flows_only) {
        const unsigned bar = bar0 + 8 * k;
        unsigned char* st = stage_ptr(k);
        mbar_expect_tx(bar, flows_only ? bytes_q : bytes_u + bytes_d + bytes_q + bytes_s);
        tma_load_4d(smem_addr(st + lay.q_off), &maps.q, x0 - QOFF, y0 - 1, p, 0, bar);
        if (!flows_only) {
            tma_load_4d(smem_addr(st + lay.u_off), &maps.u, x0, y0, p, 0, bar);
            tma_load_4d(smem_addr(st + lay.d_off), &maps.D, x0, y0, p, 0, bar);
            if (has_S) tma_load_3d(smem_addr(st + lay.s_off), &maps.S, x0, y0, p, bar);
        }
    };

    // the ring runs two planes ahead; plane p of the chunk lives in stage
    // (p - z0 + 1) % 3
    int inflight_hi = z0;
    if (t == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        issue(z0 - 1, 0, true);
        issue(z0, 1, false);
        if (z0 + 1 <= z1 && z0 + 1 < nz) {
            issue(z0 + 1, 2, false);
            inflight_hi = z0 + 1;
        }
    }
    __syncthreads();

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
    // this lane's end-label of each group and its inner node (read once:
    // lane-dependent parameter reads serialise)
    // (lf < 0: the group has no end-label for this lane)
    int lf[G], lnd[G];
    float wk[G], capl[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const bool hk = k < ng && h < tree.n[k];
        lf[k] = hk ? tree.leaf[k][h] : -1;
        lnd[k] = hk ? tree.lnode[k][h] : 0;
        wk[k] = hk ? tree.w[k][h] : 0.f;
        capl[k] = hk ? a.s_node[lnd[k]] : 0.f;
    }
    const int inn = h < ng ? tree.inner[h] : -1;  // inner node of this lane (-1: none)
    const float capi = inn >= 0 ? a.s_node[inn] : 0.f;
    // offsets in the staged u / D, flow and g planes (formed at each use)
    auto uo = [&](int k) { return lf[k] * ustride + ui; };
    auto qo = [&](int k) { return lnd[k] * (DIM * qstride) + qi; };
    auto go = [&](int k) { return lnd[k] * ustride + ui; };
    const int qo_i = (inn >= 0 ? inn : 0) * (DIM * qstride) + qi;
    const int go_i = (inn >= 0 ? inn : 0) * ustride + ui;
    // per-voxel state carried from plane p-1 to plane p: g, the flow
    // components (the z one also closes the divergence) and S
    float gprev[G], gcur[G], qxp[G], qyp[G], qzp[G];
    float gprev_i = 0.f, gcur_i = 0.f, qxp_i = 0.f, qyp_i = 0.f, qzp_i = 0.f;
    float sprev = 1.0f;
#pragma unroll
    for (int k = 0; k < G; ++k) gprev[k] = gcur[k] = qxp[k] = qyp[k] = qzp[k] = 0.f;
    bool ok = mbar_wait_bounded(bar0, 0u);
    if constexpr (DIM == 3) {
        if (ok && validE) {
            const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + lay.q_off);
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (lf[k] >= 0) qzp[k] = lds<T>(q0 + qo(k) + 2 * qstride);
            if (inn >= 0) qzp_i = lds<T>(q0 + qo_i + 2 * qstride);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        s_abort = 1;
    }
    bool bad = false;
    int p_stop = z0 - 1;
    for (int p = z0; p <= z1 && !s_abort; ++p) {
        const int s = p - z0 + 1;
        const int cs = s % 3, ps = (s + 2) % 3;
        // stage ps held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 <= z1 && p + 2 < nz) {
            issue(p + 2, ps, false);
            inflight_hi = p + 2;
        }
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + (p & 1) * g_elems;
        const float* gP = gbuf + ((p + 1) & 1) * g_elems;
        ok = true;
        if (p < nz) ok = mbar_wait_bounded(bar0 + 8 * cs, (unsigned)((s / 3) & 1));
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        float qxc[G], qyc[G], qzc[G];
#pragma unroll
        for (int k = 0; k < G; ++k) qxc[k] = qyc[k] = qzc[k] = 0.f;
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
            // (qoff: offset of the node's x component at this voxel)
            auto divergence = [&](int qoff, float& qx, float& qy, float& qz, float qzprev) {
                const T* bx = qS + qoff;
                const T* by = bx + qstride;
                qx = lds<T>(bx);
                qy = lds<T>(by);
                float dv = (qx - lds<T>(bx - 1)) + (qy - lds<T>(by - QBX));
                if constexpr (DIM == 3) {
                    qz = lds<T>(bx + 2 * qstride);
                    dv += qz - qzprev;
                }
                return dv;
            };
            float ei = 0.f;  // divergence of this lane's inner node
            if (validE && inn >= 0) ei = divergence(qo_i, qxc_i, qyc_i, qzc_i, qzp_i);
            float u[G], d[G];
            float mloc = 3.0e38f;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                // inner node k's divergence from lane k of the quad
                const float ep = __shfl_sync(0xffffffffu, ei, lane0 + k);
                u[k] = 0.f;
                d[k] = 0.f;
                if (validE && lf[k] >= 0) {
                    u[k] = lds<T>(uS + uo(k));
                    const float el = divergence(qo(k), qxc[k], qyc[k], qzc[k], qzp[k]);
                    d[k] = fmaf(wk[k], ep, dS[uo(k)] + el);
                    mloc = fminf(mloc, d[k]);
                }
            }
            float m = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
            m = fminf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            if (literal) m = 0.f;
            float sloc = 0.f;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                if (validE && lf[k] >= 0) {
                    u[k] *= ex2_approx((d[k] - m) * kexp);
                    sloc += u[k];
                }
            }
            float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            if (validE && !((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
            const float inv = rcp_fast(sum);
            // g of the end-labels (normalised, or unnormalised as printed),
            // stored labelling, and the groups' sums g_A = sum_j w_(A,j) g_j
#pragma unroll
            for (int k = 0; k < G; ++k) {
                float gk = 0.f;
                if (validE && lf[k] >= 0) {
                    const float un = u[k] * inv;
                    gk = literal ? u[k] : un;
                    gcur[k] = gk;
                    gC[go(k)] = gk;
                    if (ownerE && p < z1) stu<T>(slot_ptr<IDX32>(uout, lf[k], p, n, plane, vox), un);
                }
                float ga = wk[k] * gk;
                ga += __shfl_xor_sync(0xffffffffu, ga, 1);
                ga += __shfl_xor_sync(0xffffffffu, ga, 2);
                if (h == k) gcur_i = ga;
            }
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
            for (int k = 0; k < G; ++k)
                if (lf[k] >= 0) flow_step(lnd[k], go(k), gprev[k], gcur[k], qxp[k], qyp[k], qzp[k], capl[k]);
            if (inn >= 0) flow_step(inn, go_i, gprev_i, gcur_i, qxp_i, qyp_i, qzp_i, capi);
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            gprev[k] = gcur[k];
            qxp[k] = qxc[k];
            qyp[k] = qyc[k];
            qzp[k] = qzc[k];
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
        p_stop = p;
        if (__syncthreads_or(!ok)) {
            if (t == 0) s_abort = 1;
            break;
        }
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    if (s_abort && t == 0) {
        // bounded drain of the copies that may still be in flight: the plane
        // whose wait gave up and every plane issued after it
        for (int p = p_stop; p <= inflight_hi; ++p) {
            const int s = p - z0 + 1;
            mbar_wait_bounded(bar0 + 8 * (s % 3), (unsigned)((s / 3) & 1));
        }
    }
}

}  // namespace pfm
