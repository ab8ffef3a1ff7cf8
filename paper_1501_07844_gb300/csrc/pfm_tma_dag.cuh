// pfm_tma_dag.cuh -- TMA-pipelined fused iteration for DAG / HMF problems
// (Algorithm 2, path-weight form).
//
// Same plane pipeline as the Potts kernel (three-stage cp.async.bulk.tensor
// ring, label prox of plane p on the halo-extended tile, flow step of plane
// p-1), with a 32 x 4 tile so that three stages of every node's flow fit in
// shared memory, and four threads per voxel:
//   prox:  thread h of voxel v computes e_A = div q_A for nodes A = h, h+4, ...
//          into a per-voxel shared row, then d_j = D_j + sum_A W_(A,j) e_A for
//          end-labels j = h, h+4, ... from the sparse ancestor list of j;
//          the per-voxel minimum and normaliser are combined over the four
//          lanes with two shuffles each; the voxel's g_j then replace e in
//          the row and thread h forms g_A = sum_j W_(A,j) g_j for its nodes;
//   flow:  thread h of an owned voxel updates the flows of nodes A = h, h+4,
//          ..., from the forward differences of g_A.
// The lists hold every nonzero path weight W_(A,j) (W_(j,j) = 1), so the sums
// equal the ordered top-down / bottom-up loops of Algorithm 2 (up to the
// rounding order: the first four terms of a list are loaded together under
// predicates and summed pairwise, so a walk is not a chain of dependent
// shared-memory loads; longer lists continue in a loop); the gradient is
// linear, so differencing the accumulated g_A equals accumulating the
// end-labels' gradients.  Nodes whose capacity is zero carry no flow: the
// nodes from `nf` on (a suffix of zero-capacity nodes, e.g. the end-labels of
// the Ishikawa chain) are neither loaded, differentiated nor stored, and their
// flow buffers keep the zeros every initialisation and import leaves there.
#pragma once

#include "pfm_tma.cuh"

namespace pfm {

constexpr int DTY = 4;                         // tile rows
constexpr int DEY = DTY + 1;                   // halo-extended rows (5)
constexpr int DNE = FEX * DEY;                 // 165 halo-extended voxels
constexpr int DAG_TMA_NT = ((4 * DNE + 31) / 32) * 32;  // 672 threads
constexpr int DAG_UY = DEY;                    // u / D box rows
constexpr int DAG_QY = DEY + 1;                // flow box rows (y0-1 .. y0+4)
constexpr int DMAX = 16;                       // max end-labels / nodes
// Voxel stride of the per-voxel rows in shared memory: the rows are stored
// transposed ([entry][voxel]) with a stride = 8 (mod 32), so the four lanes
// of eight consecutive voxels touch 32 different banks.
constexpr int DAG_NV = 168;

struct DagLists {
    unsigned char anc_n[DMAX];          // ancestors of end-label j (incl. its own node)
    unsigned char anc[DMAX][DMAX];      // node ids
    float anc_w[DMAX][DMAX];            // W_(A,j)
    unsigned char desc_n[DMAX];         // end-labels below node A (incl. A itself if A is one)
    unsigned char desc[DMAX][DMAX];     // end-label indices
    float desc_w[DMAX][DMAX];           // W_(A,j)
    int nf;                             // nodes 0 .. nf-1 carry flow (1 <= nf <= nn)
};

// Shared-memory layout, sized by the runtime end-label count nl and the
// count nf of flow-carrying nodes: per stage u, D, the nf nodes' flows and S;
// two planes of g_A (nf nodes); one row of max(nl, nf) floats per voxel.
// The four lanes of a voxel read four consecutive nodes' flows at the same
// position, so the flow box is widened on the right when three stages still
// fit (qbx 44 for FP32, 56 for 16-bit types: a node stride of 24 banks mod
// 32, no two lanes on one bank), else it keeps the 32 + 2 * 16 bytes the
// halo needs (qbx 40 / 48).
struct DagTmaLayout {
    int qbx, u_off, d_off, q_off, s_off, stage_bytes, g_off, e_off, row, bar_off, total;
    __host__ __device__ static int a128(int b) { return (b + 127) / 128 * 128; }
    __host__ __device__ DagTmaLayout(int nl, int nf, int dim, int es) {
        qbx = es == 4 ? 44 : 56;
        set(nl, nf, dim, es);
        if (total + (int)sizeof(DagLists) + 64 > 227 * 1024) {
            qbx = FTX + 2 * (16 / es);
            set(nl, nf, dim, es);
        }
    }
    __host__ __device__ void set(int nl, int nf, int dim, int es) {
        u_off = 0;
        d_off = a128(nl * DAG_UY * TMA_BX * es);
        q_off = d_off + a128(nl * DAG_UY * TMA_BX * 4);
        s_off = q_off + a128(dim * nf * DAG_QY * qbx * es);
        stage_bytes = s_off + a128(FTX * DTY * 4);
        g_off = TMA_STAGES * stage_bytes;
        e_off = g_off + a128(2 * nf * DAG_UY * TMA_BX * 4);
        row = nl > nf ? nl : nf;
        bar_off = e_off + a128(DAG_NV * row * 4);
        total = bar_off + 64 + 128;
    }
};

// Stage bookkeeping carried across the tiles a CTA processes: bit k of
// `phase` is the parity of the next completion of stage k's mbarrier (every
// thread keeps it); bit k of `pending` marks a fill of stage k not yet
// waited for (thread 0 keeps it, for the drain after a timeout).
struct DagRing {
    unsigned phase = 0, pending = 0;
};

// One tile (bx, by) of z-chunk bz of one problem.  sl is the problem's lists
// in shared memory; smem the aligned dynamic shared memory; bar0 the three
// mbarriers (initialised by the caller).  Returns false after a timed-out
// wait (FLAG_TIMEOUT raised; the caller drains and stops).  Every thread of
// the CTA calls it; it ends with a CTA barrier.
template <int DIM, typename T, bool IDX32>
__device__ __forceinline__ bool dag_tma_tile(const StepArgs<DMAX, DMAX>& a, const TmaMaps& maps, const DagLists& sl,
                                             int bx, int by, int bz, unsigned char* smem, unsigned bar0,
                                             DagRing& ring) {
    constexpr int QOFF = 16 / (int)sizeof(T);
    constexpr int ustride = DAG_UY * TMA_BX;
    constexpr int PER = DMAX / 4;  // labels / nodes per thread at most
    // scalars read once (the batched kernel's arguments live in global memory)
    const int nl = a.nl, nf = sl.nf;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px, literal = a.literal, aniso = a.aniso;
    const float ctau = a.ctau;
    const DagTmaLayout lay(nl, nf, DIM, (int)sizeof(T));
    const int QBX = lay.qbx;             // flow box width (elements)
    const int qstride = DAG_QY * QBX;    // one flow component of one node
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
    const unsigned bytes_q = (unsigned)(DIM * nf * qstride * sizeof(T));
    const unsigned bytes_s = has_S ? (unsigned)(FTX * DTY * 4) : 0u;
    const float kexp = -a.inv_c * 1.4426950408889634f;
    float* gbuf = reinterpret_cast<float*>(smem + lay.g_off);
    float* ebuf = reinterpret_cast<float*>(smem + lay.e_off);
    const int g_elems = nf * ustride;

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

    // an iteration reads only the stage of its own plane (the voxel's flows
    // and S of the previous plane stay in registers): the ring runs two
    // planes ahead.  Plane p of the tile lives in stage (p - z0 + 1) % 3.
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

    // Voxel of this thread quad on the halo-extended 33 x 5 tile, owned voxels
    // first (v < 128: the 32 x 4 tile), then the y-halo row (ey = 4) and the
    // x-halo column (ex = 32).  The quad runs the prox of plane p and the flow
    // step of plane p-1 at its voxel, so g_A at its own voxel (both planes)
    // stays in registers and only the x+1 / y+1 neighbours' g_A goes through
    // shared memory: one barrier per plane.
    const bool inE = v < DNE;
    const int ex = v < FTX * DTY ? (v & (FTX - 1)) : v < FTX * DTY + FTX ? v - FTX * DTY : FTX;
    const int ey = v < FTX * DTY ? v / FTX : v < FTX * DTY + FTX ? DTY : v - (FTX * DTY + FTX);
    const int xe = x0 + ex, ye = y0 + ey;
    const bool validE = inE && xe < nx && ye < ny;
    const bool ownerE = validE && v < FTX * DTY;
    float* ecol = ebuf + (inE ? v : 0);
    const int ui = ey * TMA_BX + ex;
    const int qi = (ey + 1) * QBX + (ex + QOFF);
    const long long vox = (long long)ye * px + xe;  // slot of this voxel in its plane
    // zero steps at the last index (the g slots outside the grid hold zeros)
    const float cx = xe < nx - 1 ? ctau : 0.f;
    const float cy = ye < ny - 1 ? ctau : 0.f;

    for (int k = t; k < 2 * g_elems; k += DAG_TMA_NT) gbuf[k] = 0.f;
    // capacities of this thread's nodes, read once (lane-dependent parameter
    // reads serialise)
    // this voxel's state carried from plane p-1 to plane p: g_A, the flow
    // components of its nodes (the z one also closes the divergence) and S
    float cap[PER], gprev[PER], gcur[PER], qxp[PER], qyp[PER], qzp[PER];
    float sprev = 1.0f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        cap[i] = (h + 4 * i < nf) ? a.s_node[h + 4 * i] : 0.f;
        gprev[i] = gcur[i] = qxp[i] = qyp[i] = qzp[i] = 0.f;
    }
    // z flows of plane z0-1 (its x / y flow steps belong to the previous chunk)
    bool ok = wait_stage(0);
    if constexpr (DIM == 3) {
        if (ok && validE) {
            const T* q0 = reinterpret_cast<const T*>(stage_ptr(0) + lay.q_off);
#pragma unroll
            for (int i = 0; i < PER; ++i)
                if (h + 4 * i < nf) qzp[i] = lds<T>(q0 + ((h + 4 * i) * DIM + 2) * qstride + qi);
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
        const int s = p - z0 + 1;
        const int cs = s % 3, ps = (s + 2) % 3;
        // stage ps held plane p-1, last read before the previous barrier
        if (t == 0 && p + 2 <= z1 && p + 2 < nz) issue(p + 2, ps, false);
        unsigned char* cst = stage_ptr(cs);
        float* gC = gbuf + (p & 1) * g_elems;
        const float* gP = gbuf + ((p + 1) & 1) * g_elems;
        // each thread waits itself; a timeout reaches the CTA at the barrier
        ok = true;
        if (p < nz) ok = wait_stage(cs);
        if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
        float qxc[PER], qyc[PER], qzc[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) qxc[i] = qyc[i] = qzc[i] = 0.f;
        float scur = 1.0f;

        if (p < nz) {
            const T* uS = reinterpret_cast<const T*>(cst + lay.u_off);
            const float* dS = reinterpret_cast<const float*>(cst + lay.d_off);
            const T* qS = reinterpret_cast<const T*>(cst + lay.q_off);
            if (has_S && ownerE) scur = reinterpret_cast<const float*>(cst + lay.s_off)[ey * FTX + ex];
            // divergence of this thread's nodes (no boundary tests: the last-index
            // normal flow is an invariant zero, the box is zero-filled outside)
            if (validE) {
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int A = h + 4 * i;
                    if (A < nf) {
                        const T* qx = qS + (A * DIM + 0) * qstride + qi;
                        const T* qy = qS + (A * DIM + 1) * qstride + qi;
                        qxc[i] = lds<T>(qx);
                        qyc[i] = lds<T>(qy);
                        float dv = (qxc[i] - lds<T>(qx - 1)) + (qyc[i] - lds<T>(qy - QBX));
                        if constexpr (DIM == 3) {
                            qzc[i] = lds<T>(qS + (A * DIM + 2) * qstride + qi);
                            dv += qzc[i] - qzp[i];
                        }
                        ecol[(A) * DAG_NV] = dv;
                    }
                }
            }
            __syncwarp();
            float u[PER], d[PER];
            float mloc = 3.0e38f;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int j = h + 4 * i;
                u[i] = 0.f;
                d[i] = 0.f;
                if (validE && j < nl) {
                    u[i] = lds<T>(uS + j * ustride + ui);
                    float dj = dS[j * ustride + ui];
                    const int na = sl.anc_n[j];
                    // the first four terms unrolled under predicates (their loads
                    // issue together), the rest in a loop
                    float acc[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[k] = k < na ? sl.anc_w[j][k] * ecol[sl.anc[j][k] * DAG_NV] : 0.f;
                    dj += (acc[0] + acc[1]) + (acc[2] + acc[3]);
                    for (int k = 4; k < na; ++k) dj = fmaf(sl.anc_w[j][k], ecol[sl.anc[j][k] * DAG_NV], dj);
                    d[i] = dj;
                    mloc = fminf(mloc, dj);
                }
            }
            float m = fminf(mloc, __shfl_xor_sync(0xffffffffu, mloc, 1));
            m = fminf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            if (literal) m = 0.f;
            float sloc = 0.f;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int j = h + 4 * i;
                if (validE && j < nl) {
                    u[i] *= ex2_approx((d[i] - m) * kexp);
                    sloc += u[i];
                }
            }
            float sum = sloc + __shfl_xor_sync(0xffffffffu, sloc, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            // every lane has read its ancestors' e: the row now takes g_j
            __syncwarp();
            if (validE) {
                if (!((sum > 0.f) && (sum <= 3.0e38f))) bad = true;
                const float inv = rcp_fast(sum);

#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int j = h + 4 * i;
                    if (j < nl) {
                        const float un = u[i] * inv;
                        ecol[(j) * DAG_NV] = literal ? u[i] : un;
                        if (ownerE && p < z1) stu<T>(slot_ptr<IDX32>(uout, j, p, n, plane, vox), un);
                    }
                }
            }
            __syncwarp();
            // bottom-up accumulation g_A = sum_j W_(A,j) g_j (Algorithm 2)
            if (validE) {
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int A = h + 4 * i;
                    if (A < nf) {
                        const int nd = sl.desc_n[A];
                        float acc[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[k] = k < nd ? sl.desc_w[A][k] * ecol[sl.desc[A][k] * DAG_NV] : 0.f;
                        float g = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                        for (int k = 4; k < nd; ++k) g = fmaf(sl.desc_w[A][k], ecol[sl.desc[A][k] * DAG_NV], g);
                        gcur[i] = g;
                        gC[A * ustride + ui] = g;
                    }
                }
            }
        }

        // flow step of plane p-1 at the owned voxel: neighbours' g_A of plane
        // p-1 from shared memory (visible since the last barrier), own g_A of
        // planes p-1 and p from registers
        const int pm = p - 1;
        if (pm >= z0 && ownerE) {
            const float sf = sprev;

            const float cz = pm < nz - 1 ? ctau : 0.f;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int A = h + 4 * i;
                if (A < nf) {
                    const float* gA = gP + A * ustride + ui;
                    const float g0 = gprev[i];
                    float yv[DIM];
                    yv[0] = qxp[i] - cx * (gA[1] - g0);
                    yv[1] = qyp[i] - cy * (gA[TMA_BX] - g0);
                    if constexpr (DIM == 3) yv[2] = qzp[i] - cz * (gcur[i] - g0);
                    project_nb<DIM>(yv, cap[i] * sf, aniso);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) stv<T>(slot_ptr<IDX32>(qout, A * DIM + k, pm, n, plane, vox), yv[k]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            gprev[i] = gcur[i];
            qxp[i] = qxc[i];
            qyp[i] = qyc[i];
            qzp[i] = qzc[i];
        }
        sprev = scur;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            alive = false;
            break;
        }
    }
    if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    return alive;
}

// Bounded drain of the fills still in flight after a timed-out wait (thread 0).
__device__ __forceinline__ void dag_ring_drain(unsigned bar0, const DagRing& ring) {
    for (int k = 0; k < TMA_STAGES; ++k)
        if ((ring.pending >> k) & 1u) mbar_wait_bounded(bar0 + 8 * k, (ring.phase >> k) & 1u);
}

// Copies a problem's lists into shared memory (the four lanes of a voxel
// walk different lists; lane-dependent constant-bank reads would serialise).
__device__ __forceinline__ void dag_stage_lists(DagLists* sl, const DagLists* src) {
    static_assert(sizeof(DagLists) % 4 == 0, "lists copied as words");
    for (int k = threadIdx.x; k < (int)(sizeof(DagLists) / 4); k += DAG_TMA_NT)
        reinterpret_cast<int*>(sl)[k] = reinterpret_cast<const int*>(src)[k];
}

__device__ __forceinline__ unsigned char* dag_smem_base(unsigned char* raw) {
    return raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
}

// One problem: CTA = (x tile, y tile, z chunk).
template <int DIM, typename T, bool IDX32>
__global__ void __launch_bounds__(DAG_TMA_NT, 1)
fused_dag_tma_kernel(const StepArgs<DMAX, DMAX> a, const __grid_constant__ TmaMaps maps,
                     const __grid_constant__ DagLists lists) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ DagLists sl;
    unsigned char* smem = dag_smem_base(smem_raw);
    const DagTmaLayout lay(a.nl, lists.nf, DIM, (int)sizeof(T));
    const unsigned bar0 = smem_addr(smem + lay.bar_off);
    if (threadIdx.x == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    dag_stage_lists(&sl, &lists);
    __syncthreads();
    DagRing ring;
    if (!dag_tma_tile<DIM, T, IDX32>(a, maps, sl, blockIdx.x, blockIdx.y, blockIdx.z, smem, bar0, ring) &&
        threadIdx.x == 0)
        dag_ring_drain(bar0, ring);
}

// Many problems in one persistent launch: CTAs take (problem, x tile,
// y tile, z chunk) items in list order from a global counter (zeroed before
// the launch), so a CTA that drew short items takes more; args, maps and
// lists are per problem (this launch's parity), the maps in global memory
// (64-byte aligned, written before the launch).  The mbarrier ring carries
// over from item to item; dynamic shared memory is sized for the largest
// problem layout.
template <int DIM, typename T, bool IDX32>
__global__ void __launch_bounds__(DAG_TMA_NT, 1)
batched_dag_tma_kernel(const StepArgs<DMAX, DMAX>* __restrict__ args, const TmaMaps* __restrict__ maps,
                       const DagLists* __restrict__ lists, const int4* __restrict__ items, int n_items,
                       int bar_off, int* next_item) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ DagLists sl;
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
        // the previous item ended with a CTA barrier: s_item, sl and the
        // stages are free
        if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        dag_stage_lists(&sl, lists + w.x);
        __syncthreads();
        alive = dag_tma_tile<DIM, T, IDX32>(args[w.x], maps[w.x], sl, w.y, w.z, w.w, smem, bar0, ring);
    }
    if (!alive && threadIdx.x == 0) dag_ring_drain(bar0, ring);
}

}  // namespace pfm
