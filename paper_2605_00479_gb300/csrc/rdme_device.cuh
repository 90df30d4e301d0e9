// rdme_device.cuh -- reaction-diffusion master equation (RDME) on a lattice,
// one trajectory per GPU lane, lattice state in shared memory.
//
// The paper names the RDME (well-mixed voxels with SSA reactions, coupled by
// stochastic hops between neighbours) as the spatial setting its question
// extends to (Sec. 1, Sec. 5; future work in Sec. 6) and gives no algorithm.
// Contract (shared with the oracle, written independently):
//  * lattice nx x ny x nz, voxel v = ix + nx (iy + ny iz), reflecting
//    boundaries, hop directions -x, +x, -y, +y, -z, +z;
//  * channels of a voxel: the M reactions (the direct method's propensity
//    chain on the voxel's counts), then for each species i with D_i > 0 and
//    each existing neighbour the hop (i, dir) of value rnd(D_i' rnd(x_vi))
//    (zero below one molecule), computed once per species;
//  * voxel total = last partial sum of its channels (accumulator type);
//    totals in a binary sum tree (T = power of two >= S leaves, heap order,
//    node q = node 2q + node 2q+1 in the accumulator type), a0 = node 1;
//  * event n: uniforms and time arithmetic of the direct method; the voxel by
//    descent (left if left > r; else right with r = r - left if right > 0;
//    else left), the channel by the voxel's partial sums (first S_c > r,
//    else the last positive channel);
//  * after the event the changed voxel(s) and their ancestors are
//    recomputed; stochastic-rounding bits come from Philox counters keyed by
//    (op / 8, epoch, trajectory, 0x80000000 | v) for a voxel computed at
//    epoch e (0 initially, n + 1 after event n), (0, e, trajectory,
//    0x40000000 | q) for tree node q, and stream 1 blocks [nB, (n+1)B),
//    B = ceil((5 + log2 T) / 8), for the event-level operations (E, U2, tau,
//    target, t_new, one slot per descent level) in uniform modes;
//  * snapshots out[k][v][i][trajectory].
//
// Layout: each lane's counts, tree and epochs sit in dynamic shared memory,
// interleaved by lane (word index * blockDim + lane), so a warp's
// data-dependent accesses never conflict on a bank.
#pragma once

#include "ssa_device.cuh"

namespace ssa {

constexpr int kMaxVoxels = 1024;

struct RdmeArgs {
    RunArgs a;                 // structure, c', samples, keys, outputs, queue
    int nx, ny, nz, S, T, depth;
    double D[kMaxN];           // hop rate per direction
    const int32_t *x0_lat;     // device [S][N]
};

__host__ __device__ inline size_t rdme_align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Dynamic shared-memory layout of one block: block-wide tables, then the
// lanes' interleaved columns.
struct RdmeLayout {
    size_t smp, consts, nbmask, x, node, epoch, total;
};

__host__ __device__ inline RdmeLayout rdme_layout(int K, int S, int T, int N, int block, int elem_bytes,
                                                  bool epochs)
{
    RdmeLayout L;
    L.smp = 0;
    L.consts = rdme_align16(L.smp + (size_t)K * elem_bytes);
    L.nbmask = rdme_align16(L.consts + (size_t)(3 * kMaxM + kMaxN) * elem_bytes);
    L.x = rdme_align16(L.nbmask + (size_t)S);
    L.node = rdme_align16(L.x + (size_t)S * N * block * 4);
    L.epoch = rdme_align16(L.node + (size_t)2 * T * block * elem_bytes);
    L.total = rdme_align16(L.epoch + (epochs ? (size_t)S * block * 4 : 0));
    return L;
}

// Stochastic-rounding words keyed by (op / 8, epoch, trajectory, tag).
struct TagBits {
    uint32_t e, traj, tag, k0, k1;
    int cur;
    uint4 blk;
    __device__ __forceinline__ uint32_t word(int op)
    {
        const int b = op >> 3;
        if (b != cur) {
            blk = philox4x32_10(make_uint4((uint32_t)b, e, traj, tag), k0, k1);
            cur = b;
        }
        const int w = (op >> 1) & 3;
        return w == 0 ? blk.x : (w == 1 ? blk.y : (w == 2 ? blk.z : blk.w));
    }
};

// Rounding of a voxel's chain operations (16-bit modes) with its tag bits.
template <int PREC, int SR>
struct VoxelRounder {
    using T = ModeTraits<PREC>;
    TagBits bits;
    __device__ __forceinline__ typename T::P rnd(typename T::P x, int op)
    {
        if constexpr (T::k16) {
            if constexpr (SR != 0) return sr16<T::kFmt>(x, bits.word(op), (op & 1) != 0);
            else return rn16<T::kFmt>(x);
        } else {
            return x;
        }
    }
};

template <int PREC>
struct RLane {
    using P = typename ModeTraits<PREC>::P;
    P t, s_next;
    int64_t n, item;
    uint32_t traj, status;
    int k;
    bool active;
    uint4 blk;             // uniforms of events 2m, 2m + 1
};

// Per-block views of the shared tables and of this lane's columns.
template <int PREC>
struct RdmeView {
    using P = typename ModeTraits<PREC>::P;
    const P *smp, *cP, *h0P, *h1P, *DP;
    const uint8_t *nbmask;
    int32_t *x;            // &x_columns[lane]; element (v, i) at ((v*N + i) * bd)
    P *node;               // &node_columns[lane]; node q at (q * bd)
    uint32_t *epoch;       // &epoch_columns[lane] or null
    int bd;
    __device__ __forceinline__ int32_t &X(int v, int i, int N) const { return x[(v * N + i) * bd]; }
    __device__ __forceinline__ P &Node(int q) const { return node[q * bd]; }
};

__device__ __forceinline__ int rdme_neighbour(const RdmeArgs &A, int v, int dir)
{
    switch (dir) {
    case 0: return v - 1;
    case 1: return v + 1;
    case 2: return v - A.nx;
    case 3: return v + A.nx;
    case 4: return v - A.nx * A.ny;
    default: return v + A.nx * A.ny;
    }
}

// Voxel v at epoch e: returns its total; with sel, also the channel selected
// by residual target r.
template <int PREC, int SR>
__device__ __noinline__ typename ModeTraits<PREC>::P rdme_voxel(const RdmeArgs &A, const RdmeView<PREC> &W, int v,
                                                                uint32_t e, uint32_t traj,
                                                                typename ModeTraits<PREC>::P r, int *sel)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const RunArgs &a = A.a;
    const int N = a.N, M = a.M;
    VoxelRounder<PREC, SR> R;
    if constexpr (Tr::k16 && SR) {
        R.bits.e = e;
        R.bits.traj = traj;
        R.bits.tag = 0x80000000u | (uint32_t)v;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }
    P prop[kMaxM];
#pragma unroll 1
    for (int j = 0; j < M; ++j) {
        int op = a.chain_start[j];
        if (a.law[j] == 1) {
            const P Pv = R.rnd((P)W.X(v, a.hill_reg[j], N), op++);
            P q = Pv;
            for (int m = 1; m < a.hill_h[j]; ++m) q = R.rnd(q * Pv, op++);
            const P d = R.rnd(P(1) + q, op++);
            const P f = R.rnd(W.h1P[j] / d, op++);
            prop[j] = R.rnd(W.h0P[j] + f, op++);
        } else {
            P av = W.cP[j];
            bool zero = false;
#pragma unroll 1
            for (int i = 0; i < N; ++i) {
                const int rr = a.order[j][i];
                if (rr == 0 || a.folded[j][i]) continue;
                const int xi = W.X(v, i, N);
                zero = zero || (xi < rr);
                for (int m = 0; m < rr; ++m) {
                    const P f = R.rnd((P)(xi - m), op++);
                    av = R.rnd(av * f, op++);
                }
            }
            prop[j] = zero ? P(0) : av;
        }
    }
    const uint8_t nb = W.nbmask[v];
    const int nnb = __popc((unsigned)nb);
    P hv[kMaxN];
    int op = a.sr_ops;
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        hv[i] = P(0);
        if (nnb == 0 || !(A.D[i] > 0.0)) continue;
        const int xi = W.X(v, i, N);
        if (xi < 1) {
            op += 2;
        } else {
            const P f = R.rnd((P)xi, op++);
            hv[i] = R.rnd(W.DP[i] * f, op++);
        }
    }
    // partial sums over reactions, then hops (one per species and direction)
    const int sum_op0 = op;
    P S = P(0);
    int c = 0, mu = -1, last_pos = -1;
    auto add = [&](P val) {
        if (c == 0) S = val;
        else if constexpr (Tr::kUniform) S = R.rnd(S + val, sum_op0 + c - 1);
        else S = S + val;
        if (mu < 0 && S > r) mu = c;
        if (val > P(0)) last_pos = c;
        c += 1;
    };
#pragma unroll 1
    for (int j = 0; j < M; ++j) add(prop[j]);
    if (nnb > 0) {
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            if (!(A.D[i] > 0.0)) continue;
            for (int d = 0; d < nnb; ++d) add(hv[i]);
        }
    }
    if (sel) *sel = mu >= 0 ? mu : last_pos;
    return S;
}

template <int PREC, int SR>
__device__ __forceinline__ typename ModeTraits<PREC>::P rdme_node(const RdmeArgs &A, const RdmeView<PREC> &W, int q,
                                                                  uint32_t e, uint32_t traj)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const P s = W.Node(2 * q) + W.Node(2 * q + 1);
    if constexpr (Tr::kUniform) {
        if constexpr (SR != 0) {
            const uint4 b = philox4x32_10(make_uint4(0u, e, traj, 0x40000000u | (uint32_t)q), A.a.key0, A.a.key1);
            return sr16<Tr::kFmt>(s, b.x, false);
        } else {
            return rn16<Tr::kFmt>(s);
        }
    } else {
        return s;
    }
}

template <int PREC>
__device__ void rdme_store(const RdmeArgs &A, const RdmeView<PREC> &W, int k, int64_t item, uint32_t &status)
{
    const RunArgs &a = A.a;
    const int N = a.N;
#pragma unroll 1
    for (int v = 0; v < A.S; ++v)
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            const int64_t idx = (((int64_t)k * A.S + v) * N + i) * a.n_traj + item;
            int val = W.X(v, i, N);
            if (a.state_bytes == 2) {
                if (val > 32767) { val = 32767; status |= ST_STATE_RANGE; }
                if (val < -32768) { val = -32768; status |= ST_STATE_RANGE; }
                static_cast<int16_t *>(a.out)[idx] = (int16_t)val;
            } else {
                static_cast<int32_t *>(a.out)[idx] = val;
            }
        }
}

template <int PREC>
__device__ void rdme_finish(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L)
{
    while (L.k < A.a.K) {
        rdme_store<PREC>(A, W, L.k, L.item, L.status);
        L.k += 1;
    }
    A.a.status[L.item] = L.status;
    if (A.a.n_events) A.a.n_events[L.item] = L.n;
    if (A.a.t_final) A.a.t_final[L.item] = (double)L.t;
    L.active = false;
}

template <int PREC, int SR>
__device__ void rdme_init(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L, int64_t item)
{
    using P = typename ModeTraits<PREC>::P;
    const int N = A.a.N;
    L.item = item;
    L.traj = A.a.traj_offset + (uint32_t)item;
#pragma unroll 1
    for (int v = 0; v < A.S; ++v)
#pragma unroll 1
        for (int i = 0; i < N; ++i) W.X(v, i, N) = A.x0_lat[v * N + i];
#pragma unroll 1
    for (int v = 0; v < A.T; ++v) {
        W.Node(A.T + v) = v < A.S ? rdme_voxel<PREC, SR>(A, W, v, 0u, L.traj, P(0), nullptr) : P(0);
        if (W.epoch && v < A.S) W.epoch[v * W.bd] = 0u;
    }
#pragma unroll 1
    for (int q = A.T - 1; q >= 1; --q) W.Node(q) = rdme_node<PREC, SR>(A, W, q, 0u, L.traj);
    L.t = P(0);
    L.n = 0;
    L.k = 0;
    L.status = 0;
    L.s_next = A.a.K > 0 ? W.smp[0] : P(__int_as_float(0x7F800000));
    L.active = true;
}

// One event of an active lane (contract above).
template <int PREC, int SR>
__device__ __noinline__ void rdme_event(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L,
                                        typename ModeTraits<PREC>::P t_end)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const RunArgs &a = A.a;
    const P kInf = P(__int_as_float(0x7F800000));
    const int N = a.N, T = A.T;

    if (L.n >= a.max_events) {
        L.status |= ST_MAX_EVENTS;
        rdme_finish<PREC>(A, W, L);
        return;
    }
    const P a0 = W.Node(1);
    if (a0 != a0) { L.status |= ST_NAN; rdme_finish<PREC>(A, W, L); return; }
    if (a0 == kInf) { L.status |= ST_OVERFLOW; rdme_finish<PREC>(A, W, L); return; }
    if (a0 == P(0)) { rdme_finish<PREC>(A, W, L); return; }

    if ((L.n & 1) == 0) {
        const uint64_t blk = (uint64_t)L.n >> 1;
        L.blk = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), L.traj, 0u), a.key0, a.key1);
    }
    const uint32_t w0 = (L.n & 1) ? L.blk.z : L.blk.x;
    const uint32_t w1 = (L.n & 1) ? L.blk.w : L.blk.y;

    Rounder<PREC, SR> R;   // event-level operations (uniform modes)
    if constexpr (Tr::kUniform && SR) {
        R.bits.base = (uint64_t)L.n * (uint64_t)((5 + A.depth + 7) >> 3);
        R.bits.traj = L.traj;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }
    P tau, target, t_new;
    if constexpr (Tr::kF64) {
        const double u1 = ((double)w0 + 1.0) * 0x1p-32;
        const double u2 = (double)w1 * 0x1p-32;
        const double E = -log_f64(u1);
        tau = E / a0;
        target = u2 * a0;
        t_new = L.t + tau;
    } else {
        const float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(w1 >> 8) * 0x1p-24f;
        if constexpr (Tr::kUniform) {
            const float E = R.rnd(-log_f32(u1), 0);
            const float U2 = R.rnd(u2, 1);
            tau = R.rnd(E / a0, 2);
            target = R.rnd(U2 * a0, 3);
            t_new = R.rnd(L.t + tau, 4);
        } else {
            const float E = -log_f32(u1);
            tau = E / a0;
            target = u2 * a0;
            t_new = L.t + tau;
        }
    }
    while (L.s_next < t_new) {
        rdme_store<PREC>(A, W, L.k, L.item, L.status);
        L.k += 1;
        L.s_next = L.k < a.K ? W.smp[L.k] : kInf;
    }
    if (t_new > t_end) { rdme_finish<PREC>(A, W, L); return; }

    // voxel by descent of the sum tree
    int q = 1, level = 0;
    P r = target;
#pragma unroll 1
    while (q < T) {
        const P lf = W.Node(2 * q), rt = W.Node(2 * q + 1);
        if (lf > r) {
            q = 2 * q;
        } else if (rt > P(0)) {
            if constexpr (Tr::kUniform) r = R.rnd(r - lf, 5 + level);
            else r = r - lf;
            q = 2 * q + 1;
        } else {
            q = 2 * q;
        }
        level += 1;
    }
    const int v = q - T;
    const uint32_t ev = W.epoch ? W.epoch[v * W.bd] : 0u;
    int c = -1;
    rdme_voxel<PREC, SR>(A, W, v, ev, L.traj, r, &c);
    if (c < 0) {            // unreachable (the descent enters only positive totals); kept as a guard
        L.status |= ST_NAN;
        rdme_finish<PREC>(A, W, L);
        return;
    }

    // apply: a reaction of voxel v, or a hop v -> w
    int w = -1;
    bool negative = false;
    if (c < a.M) {
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            const int d = a.stoich[c][i];
            if (d == 0) continue;
            int &xr = W.X(v, i, N);
            xr += d;
            negative = negative || (xr < 0);
        }
    } else {
        int idx = c - a.M, species = -1, dir = -1;
        const uint8_t nb = W.nbmask[v];
        const int nnb = __popc((unsigned)nb);
#pragma unroll 1
        for (int i = 0; i < N && species < 0; ++i) {
            if (!(A.D[i] > 0.0)) continue;
            if (idx < nnb) {
                species = i;
                int seen = 0;
                for (int d = 0; d < 6; ++d) {
                    if (!((nb >> d) & 1u)) continue;
                    if (seen == idx) { dir = d; break; }
                    seen += 1;
                }
            } else {
                idx -= nnb;
            }
        }
        w = rdme_neighbour(A, v, dir);
        W.X(v, species, N) -= 1;
        W.X(w, species, N) += 1;
        negative = W.X(v, species, N) < 0;
    }
    L.t = t_new;
    L.n += 1;
    if (negative) {
        L.status |= ST_STATE_RANGE;
        rdme_finish<PREC>(A, W, L);
        return;
    }
    // recompute the changed voxels and their ancestors at epoch n + 1
    const uint32_t e = (uint32_t)L.n;
    W.Node(T + v) = rdme_voxel<PREC, SR>(A, W, v, e, L.traj, P(0), nullptr);
    if (W.epoch) W.epoch[v * W.bd] = e;
    if (w >= 0) {
        W.Node(T + w) = rdme_voxel<PREC, SR>(A, W, w, e, L.traj, P(0), nullptr);
        if (W.epoch) W.epoch[w * W.bd] = e;
    }
    int qa = (T + v) >> 1, qb = w >= 0 ? (T + w) >> 1 : 0;
#pragma unroll 1
    while (qa >= 1) {
        if (qb == qa) qb = 0;
        W.Node(qa) = rdme_node<PREC, SR>(A, W, qa, e, L.traj);
        if (qb) W.Node(qb) = rdme_node<PREC, SR>(A, W, qb, e, L.traj);
        qa >>= 1;
        qb >>= 1;
    }
}

// Persistent RDME kernel: lanes refill from the work queue; each loop
// iteration runs one event.
template <int PREC, int SR>
__global__ void __launch_bounds__(256) rdme_kernel(const __grid_constant__ RdmeArgs A)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    extern __shared__ __align__(16) unsigned char rdme_smem[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const RunArgs &a = A.a;
    constexpr bool kEpochs = Tr::k16 && SR != 0;
    const RdmeLayout lay = rdme_layout(a.K, A.S, A.T, a.N, bd, (int)sizeof(P), kEpochs);
    P *smp = reinterpret_cast<P *>(rdme_smem + lay.smp);
    P *cons = reinterpret_cast<P *>(rdme_smem + lay.consts);
    uint8_t *nbm = rdme_smem + lay.nbmask;
    for (int k = tid; k < a.K; k += bd) smp[k] = to_time<PREC>(a.samples[k]);
    for (int j = tid; j < kMaxM; j += bd) {
        const bool on = j < a.M;
        cons[j] = on ? to_prop<PREC>(a.cprime[j]) : P(0);
        cons[kMaxM + j] = on && a.law[j] == 1 ? to_prop<PREC>(a.hill_a0[j]) : P(0);
        cons[2 * kMaxM + j] = on && a.law[j] == 1 ? to_prop<PREC>(a.hill_a[j]) : P(0);
    }
    for (int i = tid; i < kMaxN; i += bd) cons[3 * kMaxM + i] = i < a.N ? to_prop<PREC>(A.D[i]) : P(0);
    for (int v = tid; v < A.S; v += bd) {
        const int ix = v % A.nx, iy = (v / A.nx) % A.ny, iz = v / (A.nx * A.ny);
        uint8_t m = 0;
        if (ix > 0) m |= 1u;
        if (ix < A.nx - 1) m |= 2u;
        if (iy > 0) m |= 4u;
        if (iy < A.ny - 1) m |= 8u;
        if (iz > 0) m |= 16u;
        if (iz < A.nz - 1) m |= 32u;
        nbm[v] = m;
    }
    __syncthreads();

    RdmeView<PREC> W;
    W.smp = smp;
    W.cP = cons;
    W.h0P = cons + kMaxM;
    W.h1P = cons + 2 * kMaxM;
    W.DP = cons + 3 * kMaxM;
    W.nbmask = nbm;
    W.x = reinterpret_cast<int32_t *>(rdme_smem + lay.x) + tid;
    W.node = reinterpret_cast<P *>(rdme_smem + lay.node) + tid;
    W.epoch = kEpochs ? reinterpret_cast<uint32_t *>(rdme_smem + lay.epoch) + tid : nullptr;
    W.bd = bd;
    const P t_end = to_time<PREC>(a.t_end);

    const unsigned lane = threadIdx.x & 31u;
    RLane<PREC> L;
    L.active = false;
    bool drained = false;
    for (;;) {
        const unsigned need = __ballot_sync(0xFFFFFFFFu, !L.active && !drained);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.queue_head, (unsigned long long)__popc(need));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (!L.active && !drained) {
                const unsigned long long item = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (item < (unsigned long long)a.n_work) rdme_init<PREC, SR>(A, W, L, (int64_t)item);
                else drained = true;
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, L.active) == 0u) break;
        if (L.active) rdme_event<PREC, SR>(A, W, L, t_end);
    }
}

}  // namespace ssa
