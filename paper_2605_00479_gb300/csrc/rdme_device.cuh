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
// data-dependent accesses never conflict on a bank.  Compiled structures
// (the StaticModel families) store only the species that change; reservoir
// species are read from a block-wide table.  The general model stores all.
#pragma once

#include <type_traits>

#include "ssa_device.cuh"

namespace ssa {

constexpr int kMaxVoxels = 1024;

struct RdmeArgs {
    RunArgs a;                 // structure, c', samples, keys, outputs, queue
    int nx, ny, nz, S, T, depth;
    int n_stored;              // species stored per voxel (see RdmeSpecies)
    double D[kMaxN];           // hop rate per direction
    const int32_t *x0_lat;     // device [S][N]
};

__host__ __device__ inline size_t rdme_align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Dynamic shared-memory layout of one block: block-wide tables, then the
// lanes' interleaved columns.
struct RdmeLayout {
    size_t smp, consts, cst, nbmask, x, node, epoch, total;
};

__host__ __device__ inline RdmeLayout rdme_layout(int K, int S, int T, int n_stored, int block, int elem_bytes,
                                                  bool epochs)
{
    RdmeLayout L;
    L.smp = 0;
    L.consts = rdme_align16(L.smp + (size_t)K * elem_bytes);
    L.cst = rdme_align16(L.consts + (size_t)(3 * kMaxM + kMaxN) * elem_bytes);
    L.nbmask = rdme_align16(L.cst + (size_t)kMaxN * 4);
    L.x = rdme_align16(L.nbmask + (size_t)S);
    L.node = rdme_align16(L.x + (size_t)S * n_stored * block * 4);
    L.epoch = rdme_align16(L.node + (size_t)2 * T * block * elem_bytes);
    L.total = rdme_align16(L.epoch + (epochs ? (size_t)S * block * 4 : 0));
    return L;
}

// Which species a lattice column holds.  General model: every species, in
// order.  Compiled structures: the non-constant species, in order.
template <class Model>
struct RdmeSpecies {
    static constexpr bool kStatic = false;
};

template <class Sx, bool NORM>
struct RdmeSpecies<StaticModel<Sx, NORM>> {
    static constexpr bool kStatic = true;
    __host__ __device__ static constexpr int count()
    {
        int c = 0;
        for (int i = 0; i < Sx::N; ++i) c += Sx::cs[i] ? 0 : 1;
        return c;
    }
    __host__ __device__ static constexpr int slot(int i)
    {
        int c = 0;
        for (int q = 0; q < i; ++q) c += Sx::cs[q] ? 0 : 1;
        return Sx::cs[i] ? -1 : c;
    }
};

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
    const int32_t *cst;    // [N] counts of the constant species (voxel 0)
    const uint8_t *nbmask;
    int32_t *x;            // &x_columns[lane]; stored species s of voxel v at ((v*ns + s) * bd)
    P *node;               // &node_columns[lane]; node q at (q * bd)
    uint32_t *epoch;       // &epoch_columns[lane] or null
    int bd, ns;
    unsigned dmask;        // bit i: species i hops (D_i > 0), so the hot path makes no binary64 compare
    __device__ __forceinline__ int32_t &at(int v, int s) const { return x[(v * ns + s) * bd]; }
    __device__ __forceinline__ P &Node(int q) const { return node[q * bd]; }
};

// Count of species I (compile time) in voxel v.
template <class Model, int I, int PREC>
__device__ __forceinline__ int rdme_get(const RdmeView<PREC> &W, int v)
{
    if constexpr (RdmeSpecies<Model>::kStatic) {
        constexpr int s = RdmeSpecies<Model>::slot(I);
        if constexpr (s < 0) return W.cst[I];
        else return W.at(v, s);
    } else {
        return W.at(v, I);
    }
}

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

// Partial sums over a voxel's channels with selection (shared by both paths).
template <int PREC, int SR>
struct ChannelSum {
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    VoxelRounder<PREC, SR> *R;
    int op0;
    P r, S;
    int c, mu, last_pos;
    __device__ __forceinline__ void add(P val)
    {
        if (c == 0) S = val;
        else if constexpr (Tr::kUniform) S = R->rnd(S + val, op0 + c - 1);
        else S = S + val;
        if (mu < 0 && S > r) mu = c;
        if (val > P(0)) last_pos = c;
        c += 1;
    }
};

// Voxel v at epoch e: returns its total; with sel, also the channel selected
// by residual target r.
template <class Model, int PREC, int SR>
__device__ __forceinline__ typename ModeTraits<PREC>::P rdme_voxel(const RdmeArgs &A, const RdmeView<PREC> &W, int v,
                                                                   uint32_t e, uint32_t traj,
                                                                   typename ModeTraits<PREC>::P r, int *sel)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const RunArgs &a = A.a;
    VoxelRounder<PREC, SR> R;
    if constexpr (Tr::k16 && SR) {
        R.bits.e = e;
        R.bits.traj = traj;
        R.bits.tag = 0x80000000u | (uint32_t)v;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }
    const uint8_t nb = W.nbmask[v];
    const int nnb = __popc((unsigned)nb);
    ChannelSum<PREC, SR> cs;
    cs.R = &R;
    cs.r = r;
    cs.S = P(0);
    cs.c = 0;
    cs.mu = -1;
    cs.last_pos = -1;

    if constexpr (RdmeSpecies<Model>::kStatic) {
        constexpr int M = Model::M, N = Model::N;
        P prop[M];
        unroll<M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            int op = Model::template chain_start<j>(a);
            if (Model::template law<j>(a) == 1) {
                const int reg = Model::template hill_reg<j>(a);
                int xr = 0;
                unroll<N>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    if (i == reg) xr = rdme_get<Model, i>(W, v);
                });
                const P Pv = R.rnd((P)xr, op++);
                P q = Pv;
                const int h = Model::template hill_h<j>(a);
                for (int m = 1; m < h; ++m) q = R.rnd(q * Pv, op++);
                const P d = R.rnd(P(1) + q, op++);
                const P f = R.rnd(W.h1P[j] / d, op++);
                prop[j] = R.rnd(W.h0P[j] + f, op++);
            } else {
                P av = W.cP[j];
                bool zero = false;
                unroll<N>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const int rr = Model::template order<j, i>(a);
                    if (rr > 0 && !Model::template folded<j, i>(a)) {
                        const int xi = rdme_get<Model, i>(W, v);
                        zero = zero || (xi < rr);
                        for (int m = 0; m < rr; ++m) {
                            const P f = R.rnd((P)(xi - m), op++);
                            av = R.rnd(av * f, op++);
                        }
                    }
                });
                prop[j] = zero ? P(0) : av;
            }
        });
        P hv[N];
        int op = Model::total_chain_ops(a);
        unroll<N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            hv[i] = P(0);
            if (nnb > 0 && ((W.dmask >> i) & 1u)) {
                const int xi = rdme_get<Model, i>(W, v);
                if (xi < 1) {
                    op += 2;
                } else {
                    const P f = R.rnd((P)xi, op++);
                    hv[i] = R.rnd(W.DP[i] * f, op++);
                }
            }
        });
        cs.op0 = op;
        unroll<M>([&](auto J) { cs.add(prop[decltype(J)::value]); });
        if (nnb > 0) {
            unroll<N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if ((W.dmask >> i) & 1u)
                    for (int d = 0; d < nnb; ++d) cs.add(hv[i]);
            });
        }
    } else {
        const int N = a.N, M = a.M;
        P prop[kMaxM];
#pragma unroll 1
        for (int j = 0; j < M; ++j) {
            int op = a.chain_start[j];
            if (a.law[j] == 1) {
                const P Pv = R.rnd((P)W.at(v, a.hill_reg[j]), op++);
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
                    const int xi = W.at(v, i);
                    zero = zero || (xi < rr);
                    for (int m = 0; m < rr; ++m) {
                        const P f = R.rnd((P)(xi - m), op++);
                        av = R.rnd(av * f, op++);
                    }
                }
                prop[j] = zero ? P(0) : av;
            }
        }
        P hv[kMaxN];
        int op = a.sr_ops;
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            hv[i] = P(0);
            if (nnb == 0 || !((W.dmask >> i) & 1u)) continue;
            const int xi = W.at(v, i);
            if (xi < 1) {
                op += 2;
            } else {
                const P f = R.rnd((P)xi, op++);
                hv[i] = R.rnd(W.DP[i] * f, op++);
            }
        }
        cs.op0 = op;
#pragma unroll 1
        for (int j = 0; j < M; ++j) cs.add(prop[j]);
        if (nnb > 0) {
#pragma unroll 1
            for (int i = 0; i < N; ++i) {
                if (!((W.dmask >> i) & 1u)) continue;
                for (int d = 0; d < nnb; ++d) cs.add(hv[i]);
            }
        }
    }
    if (sel) *sel = cs.mu >= 0 ? cs.mu : cs.last_pos;
    return cs.S;
}

// Tree node q at epoch e from its children's values (left + right).
template <int PREC, int SR>
__device__ __forceinline__ typename ModeTraits<PREC>::P rdme_sum(const RdmeArgs &A, typename ModeTraits<PREC>::P lf,
                                                                 typename ModeTraits<PREC>::P rt, int q, uint32_t e,
                                                                 uint32_t traj)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const P s = lf + rt;
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

template <int PREC, int SR>
__device__ __forceinline__ typename ModeTraits<PREC>::P rdme_node(const RdmeArgs &A, const RdmeView<PREC> &W, int q,
                                                                  uint32_t e, uint32_t traj)
{
    return rdme_sum<PREC, SR>(A, W.Node(2 * q), W.Node(2 * q + 1), q, e, traj);
}

__device__ __forceinline__ void rdme_put(const RunArgs &a, int64_t idx, int val, uint32_t &status)
{
    if (a.state_bytes == 2) {
        if (val > 32767) { val = 32767; status |= ST_STATE_RANGE; }
        if (val < -32768) { val = -32768; status |= ST_STATE_RANGE; }
        static_cast<int16_t *>(a.out)[idx] = (int16_t)val;
    } else {
        static_cast<int32_t *>(a.out)[idx] = val;
    }
}

template <class Model, int PREC>
__device__ void rdme_store(const RdmeArgs &A, const RdmeView<PREC> &W, int k, int64_t item, uint32_t &status)
{
    const RunArgs &a = A.a;
    const int N = a.N;
#pragma unroll 1
    for (int v = 0; v < A.S; ++v) {
        const int64_t base = ((int64_t)k * A.S + v) * N;
        if constexpr (RdmeSpecies<Model>::kStatic) {
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                rdme_put(a, (base + i) * a.n_traj + item, rdme_get<Model, i>(W, v), status);
            });
        } else {
#pragma unroll 1
            for (int i = 0; i < N; ++i) rdme_put(a, (base + i) * a.n_traj + item, W.at(v, i), status);
        }
    }
}

template <class Model, int PREC>
__device__ void rdme_finish(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L)
{
    while (L.k < A.a.K) {
        rdme_store<Model, PREC>(A, W, L.k, L.item, L.status);
        L.k += 1;
    }
    A.a.status[L.item] = L.status;
    if (A.a.n_events) A.a.n_events[L.item] = L.n;
    if (A.a.t_final) A.a.t_final[L.item] = (double)L.t;
    L.active = false;
}

template <class Model, int PREC, int SR>
__device__ void rdme_init(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L, int64_t item)
{
    using P = typename ModeTraits<PREC>::P;
    const int N = A.a.N;
    L.item = item;
    L.traj = A.a.traj_offset + (uint32_t)item;
#pragma unroll 1
    for (int v = 0; v < A.S; ++v) {
        if constexpr (RdmeSpecies<Model>::kStatic) {
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int s = RdmeSpecies<Model>::slot(i);
                if constexpr (s >= 0) W.at(v, s) = A.x0_lat[v * N + i];
            });
        } else {
#pragma unroll 1
            for (int i = 0; i < N; ++i) W.at(v, i) = A.x0_lat[v * N + i];
        }
    }
#pragma unroll 1
    for (int v = 0; v < A.T; ++v) {
        W.Node(A.T + v) = v < A.S ? rdme_voxel<Model, PREC, SR>(A, W, v, 0u, L.traj, P(0), nullptr) : P(0);
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

// Apply channel c of voxel v; returns the hop's destination voxel or -1.
template <class Model, int PREC>
__device__ __forceinline__ int rdme_apply(const RdmeArgs &A, const RdmeView<PREC> &W, int v, int c, bool &negative)
{
    const RunArgs &a = A.a;
    negative = false;
    if (c < a.M) {
        if constexpr (RdmeSpecies<Model>::kStatic) {
            unroll<Model::N>([&](auto I) {      // branch-free: d_i = nu[c][i] by selects
                constexpr int i = decltype(I)::value;
                constexpr int s = RdmeSpecies<Model>::slot(i);
                if constexpr (s >= 0) {
                    int d = 0;
                    bool moves = false;
                    unroll<Model::M>([&](auto J) {
                        constexpr int j = decltype(J)::value;
                        const int nu = Model::template nu<j, i>(a);
                        if (nu != 0) {
                            d = (c == j) ? nu : d;
                            moves = true;
                        }
                    });
                    if (moves) {
                        int &xr = W.at(v, s);
                        xr += d;
                        negative = negative || (xr < 0);
                    }
                }
            });
        } else {
#pragma unroll 1
            for (int i = 0; i < a.N; ++i) {
                const int d = a.stoich[c][i];
                if (d == 0) continue;
                int &xr = W.at(v, i);
                xr += d;
                negative = negative || (xr < 0);
            }
        }
        return -1;
    }
    int idx = c - a.M, species = -1, dir = -1;
    const uint8_t nb = W.nbmask[v];
    const int nnb = __popc((unsigned)nb);
#pragma unroll 1
    for (int i = 0; i < a.N && species < 0; ++i) {
        if (!((W.dmask >> i) & 1u)) continue;
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
    const int w = rdme_neighbour(A, v, dir);
    if constexpr (RdmeSpecies<Model>::kStatic) {
        unroll<Model::N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = RdmeSpecies<Model>::slot(i);
            if constexpr (s >= 0) {
                if (i == species) {
                    W.at(v, s) -= 1;
                    W.at(w, s) += 1;
                    negative = W.at(v, s) < 0;
                }
            }
        });
    } else {
        W.at(v, species) -= 1;
        W.at(w, species) += 1;
        negative = W.at(v, species) < 0;
    }
    return w;
}

// One event of an active lane (contract above).
template <class Model, int PREC, int SR>
__device__ __forceinline__ void rdme_event(const RdmeArgs &A, const RdmeView<PREC> &W, RLane<PREC> &L,
                                           typename ModeTraits<PREC>::P t_end)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const RunArgs &a = A.a;
    const P kInf = P(__int_as_float(0x7F800000));
    const int T = A.T;

    if (L.n >= a.max_events) {
        L.status |= ST_MAX_EVENTS;
        rdme_finish<Model, PREC>(A, W, L);
        return;
    }
    const P a0 = W.Node(1);
    if (a0 != a0) { L.status |= ST_NAN; rdme_finish<Model, PREC>(A, W, L); return; }
    if (a0 == kInf) { L.status |= ST_OVERFLOW; rdme_finish<Model, PREC>(A, W, L); return; }
    if (a0 == P(0)) { rdme_finish<Model, PREC>(A, W, L); return; }

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
        rdme_store<Model, PREC>(A, W, L.k, L.item, L.status);
        L.k += 1;
        L.s_next = L.k < a.K ? W.smp[L.k] : kInf;
    }
    if (t_new > t_end) { rdme_finish<Model, PREC>(A, W, L); return; }

    // voxel by descent of the sum tree, two levels per round of shared-memory
    // reads: a node's children and all four grandchildren are read together,
    // and the second level takes its pair from the grandchildren
    int q = 1, level = 0;
    P r = target;
#pragma unroll 1
    while (q < T) {
        const P lf = W.Node(2 * q), rt = W.Node(2 * q + 1);
        const bool deeper = 2 * q < T;   // children internal (then 4q + 3 <= 2T - 1)
        P g0 = P(0), g1 = P(0), g2 = P(0), g3 = P(0);
        if (deeper) {
            g0 = W.Node(4 * q);
            g1 = W.Node(4 * q + 1);
            g2 = W.Node(4 * q + 2);
            g3 = W.Node(4 * q + 3);
        }
        bool right = false;
        if (lf > r) {
            right = false;
        } else if (rt > P(0)) {
            if constexpr (Tr::kUniform) r = R.rnd(r - lf, 5 + level);
            else r = r - lf;
            right = true;
        }
        q = 2 * q + (right ? 1 : 0);
        level += 1;
        if (!deeper) break;
        const P lf2 = right ? g2 : g0, rt2 = right ? g3 : g1;
        right = false;
        if (lf2 > r) {
            right = false;
        } else if (rt2 > P(0)) {
            if constexpr (Tr::kUniform) r = R.rnd(r - lf2, 5 + level);
            else r = r - lf2;
            right = true;
        }
        q = 2 * q + (right ? 1 : 0);
        level += 1;
    }
    const int v = q - T;
    const uint32_t ev = W.epoch ? W.epoch[v * W.bd] : 0u;
    int c = -1;
    rdme_voxel<Model, PREC, SR>(A, W, v, ev, L.traj, r, &c);
    if (c < 0) {            // unreachable (the descent enters only positive totals); kept as a guard
        L.status |= ST_NAN;
        rdme_finish<Model, PREC>(A, W, L);
        return;
    }
    bool negative = false;
    const int w = rdme_apply<Model, PREC>(A, W, v, c, negative);
    L.t = t_new;
    L.n += 1;
    if (negative) {
        L.status |= ST_STATE_RANGE;
        rdme_finish<Model, PREC>(A, W, L);
        return;
    }
    // recompute the changed voxels and their ancestors at epoch n + 1.  The
    // new values climb the tree in registers; only the siblings are read from
    // shared memory, all of them before the first sum.  A sibling on the other
    // path is never read: there the two paths meet and both values are at hand.
    constexpr int kMaxDepth = 10;   // T <= kMaxVoxels = 1024
    const int depth = A.depth;
    const int la = T + v, lb = w >= 0 ? T + w : 0;
    P sa[kMaxDepth], sb[kMaxDepth];
#pragma unroll
    for (int l = 0; l < kMaxDepth; ++l) {
        sa[l] = P(0);
        sb[l] = P(0);
        if (l < depth) {
            sa[l] = W.Node((la >> l) ^ 1);
            if (lb) sb[l] = W.Node((lb >> l) ^ 1);
        }
    }
    const uint32_t e = (uint32_t)L.n;
    P va = rdme_voxel<Model, PREC, SR>(A, W, v, e, L.traj, P(0), nullptr);
    W.Node(la) = va;
    if (W.epoch) W.epoch[v * W.bd] = e;
    P vb = P(0);
    if (w >= 0) {
        vb = rdme_voxel<Model, PREC, SR>(A, W, w, e, L.traj, P(0), nullptr);
        W.Node(lb) = vb;
        if (W.epoch) W.epoch[w * W.bd] = e;
    }
    int qa = la, qb = lb;
#pragma unroll
    for (int l = 0; l < kMaxDepth; ++l) {
        if (l >= depth) break;
        const int pa = qa >> 1;
        if (qb != 0 && (qb >> 1) == pa) {            // the paths meet at pa
            const P lf = (qa & 1) ? vb : va, rt = (qa & 1) ? va : vb;
            va = rdme_sum<PREC, SR>(A, lf, rt, pa, e, L.traj);
            qb = 0;
        } else {
            const P lf = (qa & 1) ? sa[l] : va, rt = (qa & 1) ? va : sa[l];
            va = rdme_sum<PREC, SR>(A, lf, rt, pa, e, L.traj);
            if (qb != 0) {
                const int pb = qb >> 1;
                const P lfb = (qb & 1) ? sb[l] : vb, rtb = (qb & 1) ? vb : sb[l];
                vb = rdme_sum<PREC, SR>(A, lfb, rtb, pb, e, L.traj);
                W.Node(pb) = vb;
                qb = pb;
            }
        }
        W.Node(pa) = va;
        qa = pa;
    }
}

// Persistent RDME kernel: lanes refill from the work queue; each loop
// iteration runs up to kRdmeSlice events per lane.
constexpr int kRdmeSlice = 8;

template <class Model, int PREC, int SR>
__global__ void __launch_bounds__(256) rdme_kernel(const __grid_constant__ RdmeArgs A)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    extern __shared__ __align__(16) unsigned char rdme_smem[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const RunArgs &a = A.a;
    constexpr bool kEpochs = Tr::k16 && SR != 0;
    const RdmeLayout lay = rdme_layout(a.K, A.S, A.T, A.n_stored, bd, (int)sizeof(P), kEpochs);
    P *smp = reinterpret_cast<P *>(rdme_smem + lay.smp);
    P *cons = reinterpret_cast<P *>(rdme_smem + lay.consts);
    int32_t *cst = reinterpret_cast<int32_t *>(rdme_smem + lay.cst);
    uint8_t *nbm = rdme_smem + lay.nbmask;
    for (int k = tid; k < a.K; k += bd) smp[k] = to_time<PREC>(a.samples[k]);
    for (int j = tid; j < kMaxM; j += bd) {
        const bool on = j < a.M;
        cons[j] = on ? to_prop<PREC>(a.cprime[j]) : P(0);
        cons[kMaxM + j] = on && a.law[j] == 1 ? to_prop<PREC>(a.hill_a0[j]) : P(0);
        cons[2 * kMaxM + j] = on && a.law[j] == 1 ? to_prop<PREC>(a.hill_a[j]) : P(0);
    }
    for (int i = tid; i < kMaxN; i += bd) {
        cons[3 * kMaxM + i] = i < a.N ? to_prop<PREC>(A.D[i]) : P(0);
        cst[i] = i < a.N ? A.x0_lat[i] : 0;
    }
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
    W.cst = cst;
    W.nbmask = nbm;
    W.x = reinterpret_cast<int32_t *>(rdme_smem + lay.x) + tid;
    W.node = reinterpret_cast<P *>(rdme_smem + lay.node) + tid;
    W.epoch = kEpochs ? reinterpret_cast<uint32_t *>(rdme_smem + lay.epoch) + tid : nullptr;
    W.bd = bd;
    W.ns = A.n_stored;
    W.dmask = 0u;
    for (int i = 0; i < kMaxN; ++i)
        if (i < a.N && A.D[i] > 0.0) W.dmask |= 1u << i;
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
                if (item < (unsigned long long)a.n_work) rdme_init<Model, PREC, SR>(A, W, L, (int64_t)item);
                else drained = true;
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, L.active) == 0u) break;
        // several events between refill checks (a lane that finishes idles
        // until the slice ends)
#pragma unroll 1
        for (int sl = 0; sl < kRdmeSlice; ++sl)
            if (L.active) rdme_event<Model, PREC, SR>(A, W, L, t_end);
    }
}

// Threads per block: the largest multiple of 32 (at most max_block) whose
// columns fit in the opt-in shared memory of one block; 0 if none does.
inline int rdme_block_size_for(const RdmeArgs &A, int elem_bytes, bool epochs, int max_block, size_t smem_limit)
{
    int block = (max_block / 32) * 32;
    while (block >= 32 && rdme_layout(A.a.K, A.S, A.T, A.n_stored, block, elem_bytes, epochs).total > smem_limit)
        block -= 32;
    return block < 32 ? 0 : block;
}

template <class Model, int PREC, int SR>
cudaError_t rdme_launch_mode(const RdmeArgs &A, int max_block, int blocks_per_sm, size_t smem_limit,
                             cudaStream_t stream, int *grid_out, int *block_out)
{
    using P = typename ModeTraits<PREC>::P;
    constexpr bool kEpochs = ModeTraits<PREC>::k16 && SR != 0;
    auto k = rdme_kernel<Model, PREC, SR>;
    const int block = rdme_block_size_for(A, (int)sizeof(P), kEpochs, max_block, smem_limit);
    if (block < 32) return cudaErrorInvalidConfiguration;
    const size_t bytes = rdme_layout(A.a.K, A.S, A.T, A.n_stored, block, (int)sizeof(P), kEpochs).total;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = (A.a.n_work + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    *block_out = block;
    k<<<(unsigned)grid, (unsigned)block, bytes, stream>>>(A);
    return cudaGetLastError();
}

// All (precision, rounding) instantiations of one model structure.
template <class Model>
cudaError_t rdme_launch_model(const RdmeArgs &A, int prec, int sr, int max_block, int blocks_per_sm,
                              size_t smem_limit, cudaStream_t s, int *grid, int *block)
{
    switch (prec) {
    case FP64: return rdme_launch_mode<Model, FP64, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    case FP32: return rdme_launch_mode<Model, FP32, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    case MIXED_F16:
        return sr ? rdme_launch_mode<Model, MIXED_F16, 1>(A, max_block, blocks_per_sm, smem_limit, s, grid, block)
                  : rdme_launch_mode<Model, MIXED_F16, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    case MIXED_BF16:
        return sr ? rdme_launch_mode<Model, MIXED_BF16, 1>(A, max_block, blocks_per_sm, smem_limit, s, grid, block)
                  : rdme_launch_mode<Model, MIXED_BF16, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    case UNIFORM_F16:
        return sr ? rdme_launch_mode<Model, UNIFORM_F16, 1>(A, max_block, blocks_per_sm, smem_limit, s, grid, block)
                  : rdme_launch_mode<Model, UNIFORM_F16, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    case UNIFORM_BF16:
        return sr ? rdme_launch_mode<Model, UNIFORM_BF16, 1>(A, max_block, blocks_per_sm, smem_limit, s, grid, block)
                  : rdme_launch_mode<Model, UNIFORM_BF16, 0>(A, max_block, blocks_per_sm, smem_limit, s, grid, block);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssa
