// Device kernels of the FPSA source iteration (arXiv:1907.13013), templated on
// the arithmetic type T (double for the FP64 path, float for the inner solves of
// the mixed-precision path).
//
// Data layout in HBM (last index contiguous):
//   angular / nodal arrays   X[r][g][a][n]   r < R, g < sumK, a in {0=L,1=R}, n < N
//   moment arrays            P[r][g][a][l]   l padded to N (l >= L+1 unused or 0)
//   sweep coefficients       coef[g][6][n]
//   FP blocks                A[g][2N][2N]    row-major, replaced in place by the
//                                            TRANSPOSED inverse when g is eliminated
//   upwind couplings         Bc/Cc[slot][N/2][N/2]
// The 2N unknowns of a cell are [u_L(0..N-1), u_R(0..N-1)] with ordinates
// ascending, so the index sets of the LD upwind coupling are
//   L- = [0, N/2)  L+ = [N/2, N)  R- = [N, 3N/2)  R+ = [3N/2, 2N)
// (L+ and R- receive inflow from the neighbours, R+ and L- are the outflows).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fpsa_internal.h"
#include "bulk_copy.cuh"

namespace cg = cooperative_groups;

namespace fpsa {

// ---------------------------------------------------------------------------
// LD cell algebra (Sec. 2.2 reading: Galerkin LD, consistent mass, upwind).
// For ordinate mu with nu = |mu|, the upwind node u (L for mu>0, R for mu<0)
// and the downwind node d, one cell solves
//   [[nu/2 + s h/3, nu/2 + s h/6], [-nu/2 + s h/6, nu/2 + s h/3]] [psi_u, psi_d]
//       = m [q_u, q_d] + [nu psi_in, 0],    m = (h/6)[[2,1],[1,2]].
// Its solution is affine in (q_u, q_d, psi_in):
//   psi_u = G_uu q_u + G_ud q_d + a_u psi_in
//   psi_d = G_du q_u + G_dd q_d + alpha psi_in
// alpha = (6 - 2 tau)/(6 + 4 tau + tau^2), tau = s h / nu, is the cell
// transmission (the [1/2] Pade approximant of exp(-tau)). The coefficients are
// computed once per cross-section set in FP64 and stored as coef[g][k][n] with
// k = 0 alpha, 1 a_u, 2 G_uu, 3 G_ud, 4 G_du, 5 G_dd.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sweep_coef(const double *__restrict__ mu, const double *__restrict__ h,
                             const double *__restrict__ sigma_t, int N, int sumK, T *__restrict__ coef) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)sumK * N) return;
    int g = (int)(idx / N), n = (int)(idx - (size_t)g * N);
    double nu = fabs(mu[n]), hh = h[g], sh = sigma_t[g] * hh;
    double T00 = 0.5 * nu + sh / 3.0, T01 = 0.5 * nu + sh / 6.0, T10 = -0.5 * nu + sh / 6.0, T11 = T00;
    double id = 1.0 / (T00 * T11 - T01 * T10);
    double I00 = T11 * id, I01 = -T01 * id, I10 = -T10 * id, I11 = T00 * id;
    double m0 = hh / 3.0, m1 = hh / 6.0;
    T *c = coef + (size_t)g * 6 * N + n;
    c[0] = (T)(I10 * nu);
    c[N] = (T)(I00 * nu);
    c[2 * N] = (T)(I00 * m0 + I01 * m1);
    c[3 * N] = (T)(I00 * m1 + I01 * m0);
    c[4 * N] = (T)(I10 * m0 + I11 * m1);
    c[5 * N] = (T)(I10 * m1 + I11 * m0);
}

// ---------------------------------------------------------------------------
// Transport sweep L psi = q (Eq. trsi / Eq. predict), one block per
// (ordinate, instance, rhs). The sequential recurrence over cells
// x_{k+1} = alpha_k x_k + beta_k (x = outflow of cell k, beta_k its outflow
// for zero inflow) is an affine map per cell; affine maps compose
// associatively, so each thread composes the maps of a contiguous chunk of
// cells (pass 1), the block scans the chunk maps (warp shuffles, then across
// warps), and each thread re-sweeps its chunk from the exact inflow (pass 2).
//
// Edge inflow x0 of ordinate n (upwind edge s: left for mu > 0):
//   vacuum edge       x0 = psi_inc[r][b][s][n] (given incoming flux; 0 if none)
//   reflective edge   x0 = outflow at s of the mirror ordinate n' = N-1-n. With the
//                     whole-slab maps x -> A x + E of n and n' for zero inflow
//                     (the totals pass, kTotals = true, writes them to tot), this is
//                     A' x0' + E' with x0' the inflow of n' at the far edge: its
//                     given flux, or, if that edge reflects too, A x0 + E, so that
//                     x0 = (A' E + E') / (1 - A A')  (|A A'| < 1 for sigma_t > 0).
// The mirror-ordinate coupling is thus exact per sweep (no lagged edge values).
// ---------------------------------------------------------------------------
template <typename T>
struct Affine {
    T a, b;  // x -> a x + b
};

template <typename T>
__device__ __forceinline__ Affine<T> compose(Affine<T> first, Affine<T> then) {
    return {then.a * first.a, then.a * first.b + then.b};
}

constexpr int32_t kBcReflect = 1;

constexpr int kSweepBatch = 8;  // cells whose inputs one thread requests together

template <typename T, int NT, bool kTotals = false>
__global__ void __launch_bounds__(NT) k_sweep(const T *__restrict__ q, T *__restrict__ psi,
                                              const T *__restrict__ coef, const double *__restrict__ mu,
                                              const int32_t *__restrict__ off, const int32_t *__restrict__ Kc,
                                              int N, int sumK, const T *__restrict__ psi_inc = nullptr,
                                              const int32_t *__restrict__ bc = nullptr, T *__restrict__ tot = nullptr) {
    __shared__ Affine<T> warp_tot[NT / 32];
    const int n = blockIdx.x, b = blockIdx.y, r = blockIdx.z, B = gridDim.y;
    const int K = Kc[b], o = off[b];
    const bool fwd = mu[n] > 0.0;
    const int nu_ = fwd ? 0 : 1, nd_ = 1 - nu_;
    const int chunk = (K + NT - 1) / NT;
    const int p0 = min((int)threadIdx.x * chunk, K), p1 = min(p0 + chunk, K);
    const size_t base = ((size_t)r * sumK + o) * 2 * N + n;
    const T *qb = q + base;
    T *pb_ = psi + base;
    const T *cb = coef + (size_t)o * 6 * N + n;

    // pass 1: the chunk's affine map, inputs requested kSweepBatch cells at a time
    // (all loads of a batch in flight together, then the dependent recurrence)
    Affine<T> m{T(1), T(0)};
    for (int pb = p0; pb < p1; pb += kSweepBatch) {
        T qu[kSweepBatch], qd[kSweepBatch], al[kSweepBatch], gdu[kSweepBatch], gdd[kSweepBatch];
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t) {
            const int p = pb + t;
            if (p < p1) {
                const int c = fwd ? p : K - 1 - p;
                const T *cc = cb + (size_t)c * 6 * N;
                qu[t] = qb[(size_t)(2 * c + nu_) * N];
                qd[t] = qb[(size_t)(2 * c + nd_) * N];
                al[t] = cc[0];
                gdu[t] = cc[4 * N];
                gdd[t] = cc[5 * N];
            }
        }
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t)
            if (pb + t < p1) {
                m.b = al[t] * m.b + (gdu[t] * qu[t] + gdd[t] * qd[t]);
                m.a = al[t] * m.a;
            }
    }
    // inclusive scan over the block (thread order = sweep order)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Affine<T> inc = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T pa = __shfl_up_sync(0xffffffffu, inc.a, d);
        T pbv = __shfl_up_sync(0xffffffffu, inc.b, d);
        if (lane >= d) inc = compose(Affine<T>{pa, pbv}, inc);
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        Affine<T> t = (lane < NT / 32) ? warp_tot[lane] : Affine<T>{T(1), T(0)};
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T pa = __shfl_up_sync(0xffffffffu, t.a, d);
            T pbv = __shfl_up_sync(0xffffffffu, t.b, d);
            if (lane >= d) t = compose(Affine<T>{pa, pbv}, t);
        }
        if (lane < NT / 32) warp_tot[lane] = t;  // inclusive prefix over warps
    }
    __syncthreads();
    if (kTotals) {
        if (threadIdx.x == 0) {
            const Affine<T> t = warp_tot[NT / 32 - 1];
            T *o = tot + (((size_t)r * B + b) * N + n) * 2;
            o[0] = t.a;
            o[1] = t.b;
        }
        return;
    }
    // inflow at the upwind edge
    const int s = fwd ? 0 : 1;
    const size_t ib = (size_t)r * B + b;
    T x0 = psi_inc ? psi_inc[(ib * 2 + s) * N + n] : T(0);
    if (bc && bc[2 * b + s] == kBcReflect) {
        const int nm = N - 1 - n;
        const T *tn = tot + (ib * N + n) * 2, *tm = tot + (ib * N + nm) * 2;
        if (bc[2 * b + 1 - s] == kBcReflect) {
            x0 = (tm[0] * tn[1] + tm[1]) / (T(1) - tn[0] * tm[0]);
        } else {
            const T far = psi_inc ? psi_inc[(ib * 2 + 1 - s) * N + nm] : T(0);
            x0 = tm[0] * far + tm[1];
        }
    }
    // exclusive prefix for this thread, applied to the inflow x0
    T before_warp = (wid > 0) ? warp_tot[wid - 1].a * x0 + warp_tot[wid - 1].b : x0;
    T inc_b_full = inc.a * before_warp + inc.b;  // inclusive, thread-level
    T x = __shfl_up_sync(0xffffffffu, inc_b_full, 1);
    if (lane == 0) x = before_warp;

    // pass 2: re-sweep the chunk from its exact inflow, in batches as in pass 1
    for (int pb = p0; pb < p1; pb += kSweepBatch) {
        T qu[kSweepBatch], qd[kSweepBatch], cf[6][kSweepBatch];
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t) {
            const int p = pb + t;
            if (p < p1) {
                const int c = fwd ? p : K - 1 - p;
                const T *cc = cb + (size_t)c * 6 * N;
                qu[t] = qb[(size_t)(2 * c + nu_) * N];
                qd[t] = qb[(size_t)(2 * c + nd_) * N];
#pragma unroll
                for (int k = 0; k < 6; ++k) cf[k][t] = cc[(size_t)k * N];
            }
        }
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t) {
            const int p = pb + t;
            if (p < p1) {
                const int c = fwd ? p : K - 1 - p;
                // cf: 0 alpha, 1 a_u, 2 G_uu, 3 G_ud, 4 G_du, 5 G_dd
                const T pu = cf[2][t] * qu[t] + cf[3][t] * qd[t] + cf[1][t] * x;
                const T pd = cf[4][t] * qu[t] + cf[5][t] * qd[t] + cf[0][t] * x;
                pb_[(size_t)(2 * c + nu_) * N] = pu;
                pb_[(size_t)(2 * c + nd_) * N] = pd;
                x = pd;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Segmented transport sweep (the same recurrence, maps and edge inflows as
// k_sweep), laid out for coalesced access: a block holds 32 ordinates of one
// direction in its lanes (consecutive n: one 128-byte line per cell value) and
// kSegWarps chunks of cpt consecutive cells (in sweep order) in its warps, so a
// segment covers kSegWarps * cpt cells and a (direction, 32-ordinate group,
// instance, rhs) is swept by nseg blocks along the slab (nseg <= kSegMax):
//   k_sweep_maps   each chunk's affine map (x -> a x + b for the chunk's outflow)
//                  and their composition over the segment, written per ordinate;
//   k_sweep_apply  the segment's inflow: the edge inflow (as in k_sweep, the
//                  whole-slab maps of n and of its mirror composed from all
//                  segment maps at a reflective edge) carried through the maps of
//                  the segments before it, then through the chunk maps before
//                  the warp's chunk; then the chunk is re-swept from that inflow.
// Maps are stored as (a, b) pairs: cmap[zb][seg][warp][n], smap[zb][seg][n].
// ---------------------------------------------------------------------------
constexpr int kSegWarps = 8, kSegMax = 64;
static_assert(kSegMax % kSegWarps == 0, "segment maps split evenly over the warps");

struct SweepLane {
    int n, K, o, r, b;
    bool valid, fwd;
};

__device__ __forceinline__ SweepLane sweep_lane(int N, const int32_t *off, const int32_t *Kc, int B) {
    SweepLane s;
    const int gpd = (N / 2 + 31) / 32;
    const int d = blockIdx.x / gpd, idx = (blockIdx.x % gpd) * 32 + (threadIdx.x & 31);
    s.valid = idx < N / 2;
    s.fwd = d == 1;  // ordinates n >= N/2 have mu > 0: swept left to right
    s.n = d ? N / 2 + idx : idx;
    s.b = blockIdx.z % B;
    s.r = blockIdx.z / B;
    s.K = Kc[s.b];
    s.o = off[s.b];
    return s;
}

template <typename T>
__device__ __forceinline__ Affine<T> load_map(const T *m, size_t i) {
    return {__ldcg(m + 2 * i), __ldcg(m + 2 * i + 1)};
}

template <typename T>
__global__ void __launch_bounds__(kSegWarps * 32) k_sweep_maps(const T *__restrict__ q, const T *__restrict__ coef,
                                                               const int32_t *__restrict__ off,
                                                               const int32_t *__restrict__ Kc, int N, int sumK, int B,
                                                               int cpt, int nseg, T *__restrict__ cmap,
                                                               T *__restrict__ smap) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    __shared__ Affine<T> part[kSegWarps][32];
    const SweepLane L = sweep_lane(N, off, Kc, B);
    const int seg = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg_len = kSegWarps * cpt;
    if (seg * seg_len >= L.K) return;  // whole block: segments beyond this instance's cells
    const int nu_ = L.fwd ? 0 : 1, nd_ = 1 - nu_;
    const int p0 = seg * seg_len + w * cpt, p1 = min(p0 + cpt, L.K);
    Affine<T> m{T(1), T(0)};
    if (L.valid) {
        const T *qb = q + ((size_t)L.r * sumK + L.o) * 2 * N + L.n;
        const T *cb = coef + (size_t)L.o * 6 * N + L.n;
        for (int pb = p0; pb < p1; pb += kSweepBatch) {
            T qu[kSweepBatch], qd[kSweepBatch], al[kSweepBatch], gdu[kSweepBatch], gdd[kSweepBatch];
#pragma unroll
            for (int t = 0; t < kSweepBatch; ++t) {
                const int p = pb + t;
                if (p < p1) {
                    const int c = L.fwd ? p : L.K - 1 - p;
                    const T *cc = cb + (size_t)c * 6 * N;
                    qu[t] = qb[(size_t)(2 * c + nu_) * N];
                    qd[t] = qb[(size_t)(2 * c + nd_) * N];
                    al[t] = cc[0];
                    gdu[t] = cc[4 * N];
                    gdd[t] = cc[5 * N];
                }
            }
#pragma unroll
            for (int t = 0; t < kSweepBatch; ++t)
                if (pb + t < p1) {
                    m.b = al[t] * m.b + (gdu[t] * qu[t] + gdd[t] * qd[t]);
                    m.a = al[t] * m.a;
                }
        }
        const size_t ci = (((size_t)blockIdx.z * nseg + seg) * kSegWarps + w) * N + L.n;
        cmap[2 * ci] = m.a;
        cmap[2 * ci + 1] = m.b;
    }
    part[w][lane] = m;
    __syncthreads();
    if (w == 0 && L.valid) {
        Affine<T> t = part[0][lane];
        for (int v = 1; v < kSegWarps; ++v) t = compose(t, part[v][lane]);
        const size_t si = ((size_t)blockIdx.z * nseg + seg) * N + L.n;
        smap[2 * si] = t.a;
        smap[2 * si + 1] = t.b;
    }
}

// Composition of the segment maps [s0, s1) of ordinate n (in sweep order), split over
// the block's warps (contiguous ranges, then combined in order by warp 0; the result
// is in part[0][lane] after the block barrier). All threads call it.
template <typename T>
__device__ __forceinline__ void compose_segments(const T *smap, int zb, int nseg, int N, int n, bool valid, int s0,
                                                 int s1, Affine<T> (*part)[32]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kPer = kSegMax / kSegWarps;  // segment maps per warp (all requested at once)
    const int cnt = max(s1 - s0, 0), per = (cnt + kSegWarps - 1) / kSegWarps;
    const int a0 = s0 + w * per, a1 = min(s1, a0 + per);
    Affine<T> m{T(1), T(0)};
    if (valid) {
        Affine<T> v[kPer];
#pragma unroll
        for (int t = 0; t < kPer; ++t)
            v[t] = (a0 + t < a1) ? load_map(smap, ((size_t)zb * nseg + a0 + t) * N + n) : Affine<T>{T(1), T(0)};
#pragma unroll
        for (int t = 0; t < kPer; ++t) m = compose(m, v[t]);
    }
    __syncthreads();  // part may still be read from a previous use
    part[w][lane] = m;
    __syncthreads();
    if (w == 0) {
        Affine<T> t = part[0][lane];
        for (int v = 1; v < kSegWarps; ++v) t = compose(t, part[v][lane]);
        part[0][lane] = t;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kSegWarps * 32) k_sweep_apply(const T *__restrict__ q, T *__restrict__ psi,
                                                                const T *__restrict__ coef,
                                                                const int32_t *__restrict__ off,
                                                                const int32_t *__restrict__ Kc, int N, int sumK, int B,
                                                                int cpt, int nseg, const T *__restrict__ cmap,
                                                                const T *__restrict__ smap,
                                                                const T *__restrict__ psi_inc,
                                                                const int32_t *__restrict__ bc) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    __shared__ Affine<T> part[kSegWarps][32];
    __shared__ T xin[32];
    const SweepLane L = sweep_lane(N, off, Kc, B);
    const int seg = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31, zb = blockIdx.z;
    const int seg_len = kSegWarps * cpt;
    if (seg * seg_len >= L.K) return;  // whole block
    const int ns = (L.K + seg_len - 1) / seg_len;  // this instance's segments
    // edge inflow of ordinate n at its upwind edge s
    const int s = L.fwd ? 0 : 1;
    const size_t ib = (size_t)L.r * B + L.b;
    T x0 = (psi_inc && L.valid) ? psi_inc[(ib * 2 + s) * N + L.n] : T(0);
    if (bc && bc[2 * L.b + s] == kBcReflect) {
        // whole-slab maps of n and of its mirror nm (the mirror's lanes sit in the
        // other direction's blocks; its segment maps are read from smap)
        const int nm = N - 1 - L.n;
        compose_segments(smap, zb, nseg, N, L.n, L.valid, 0, ns, part);
        const Affine<T> tn = part[0][lane];
        compose_segments(smap, zb, nseg, N, nm, L.valid, 0, ns, part);
        const Affine<T> tm = part[0][lane];
        if (bc[2 * L.b + 1 - s] == kBcReflect) {
            x0 = (tm.a * tn.b + tm.b) / (T(1) - tn.a * tm.a);
        } else {
            const T far = (psi_inc && L.valid) ? psi_inc[(ib * 2 + 1 - s) * N + nm] : T(0);
            x0 = tm.a * far + tm.b;
        }
    }
    // inflow of this segment, then of this warp's chunk
    compose_segments(smap, zb, nseg, N, L.n, L.valid, 0, seg, part);
    if (w == 0) xin[lane] = part[0][lane].a * x0 + part[0][lane].b;
    __syncthreads();
    T x = xin[lane];
    if (!L.valid) return;
    {
        Affine<T> cm[kSegWarps - 1];
#pragma unroll
        for (int v = 0; v < kSegWarps - 1; ++v)
            cm[v] = v < w ? load_map(cmap, (((size_t)zb * nseg + seg) * kSegWarps + v) * N + L.n) : Affine<T>{T(1), T(0)};
#pragma unroll
        for (int v = 0; v < kSegWarps - 1; ++v) x = cm[v].a * x + cm[v].b;
    }
    // re-sweep the chunk from its exact inflow
    const int nu_ = L.fwd ? 0 : 1, nd_ = 1 - nu_;
    const int p0 = seg * seg_len + w * cpt, p1 = min(p0 + cpt, L.K);
    const size_t base = ((size_t)L.r * sumK + L.o) * 2 * N + L.n;
    const T *qb = q + base;
    T *pb_ = psi + base;
    const T *cb = coef + (size_t)L.o * 6 * N + L.n;
    for (int pb = p0; pb < p1; pb += kSweepBatch) {
        T qu[kSweepBatch], qd[kSweepBatch], cf[6][kSweepBatch];
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t) {
            const int p = pb + t;
            if (p < p1) {
                const int c = L.fwd ? p : L.K - 1 - p;
                const T *cc = cb + (size_t)c * 6 * N;
                qu[t] = qb[(size_t)(2 * c + nu_) * N];
                qd[t] = qb[(size_t)(2 * c + nd_) * N];
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) cf[kk][t] = cc[(size_t)kk * N];
            }
        }
#pragma unroll
        for (int t = 0; t < kSweepBatch; ++t) {
            const int p = pb + t;
            if (p < p1) {
                const int c = L.fwd ? p : L.K - 1 - p;
                // cf: 0 alpha, 1 a_u, 2 G_uu, 3 G_ud, 4 G_du, 5 G_dd
                const T pu = cf[2][t] * qu[t] + cf[3][t] * qd[t] + cf[1][t] * x;
                const T pd = cf[4][t] * qu[t] + cf[5][t] * qd[t] + cf[0][t] * x;
                pb_[(size_t)(2 * c + nu_) * N] = pu;
                pb_[(size_t)(2 * c + nd_) * N] = pd;
                x = pd;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Angular contractions. Ys[c][o] = sum_k MatT[k][o] Xs[c][k] over the columns
// c < ncols of a shared-memory tile; MatT is the transposed operator in global
// memory (k-major, so consecutive threads read consecutive o).
//   moments    phi_l = sum_n D[l][n] psi_n            (Eq. phi-mom)   MatT = D^T
//   expansion  q_n = sum_l M[n][l] (sigma_{s,l} phi_l + Q_l)  (Eq. treq) MatT = M^T
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void block_contract(const T *Xs, int ldx, const T *__restrict__ MatT, int N, int ncols,
                                               T *Ys, int ldy, const T *__restrict__ add = nullptr) {
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, o = idx - c * N;
        const T *x = Xs + c * ldx;
        T acc = add ? add[(size_t)c * ldy + o] : T(0);
#pragma unroll 8
        for (int k = 0; k < N; ++k) acc = fma(MatT[(size_t)k * N + o], x[k], acc);
        Ys[c * ldy + o] = acc;
    }
}

// Columns handled by one contraction block: CB cells x 2 nodes.
constexpr int kContractCells = 8;

// q = M (sigma_s phi + Q) + q_ang for every column (Eq. treq: scattering + external
// source given as moments Q and/or as nodal angular values q_ang; either may be NULL).
template <typename T>
__global__ void k_scatter(const T *__restrict__ phi, const T *__restrict__ sigma_s, const T *__restrict__ Qext,
                          const T *__restrict__ MT, T *__restrict__ q, int N, int sumK,
                          const T *__restrict__ Qang = nullptr) {
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncell = min(kContractCells, sumK - g0);
    const int ncols = 2 * ncell;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        const int g = g0 + c / 2;
        const size_t e = (colbase + c) * N + l;
        Xs[c * N + l] = sigma_s[(size_t)g * N + l] * phi[e] + (Qext ? Qext[e] : T(0));
    }
    __syncthreads();
    block_contract(Xs, N, MT, N, ncols, q + colbase * N, N, Qang ? Qang + colbase * N : nullptr);
}

// FPSA, after the sweep: phi_half = D psi_half; then the FP right-hand side
// m (x) M diag(sigma_s) (phi_half - phi)  (Eq. correct: S (psi^{m+1/2} - psi^m),
// mass-weighted for the LD system).
template <typename T>
__global__ void k_fp_rhs(const T *__restrict__ psi_half, const T *__restrict__ phi, T *__restrict__ phi_half,
                         const T *__restrict__ sigma_s, const double *__restrict__ h, const T *__restrict__ DT,
                         const T *__restrict__ MT, T *__restrict__ rhs, int N, int sumK) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    T *Ys = Xs + 2 * kContractCells * N;
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncell = min(kContractCells, sumK - g0);
    const int ncols = 2 * ncell;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) Xs[idx] = psi_half[colbase * N + idx];
    __syncthreads();
    block_contract(Xs, N, DT, N, ncols, Ys, N);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        const int g = g0 + c / 2;
        const T ph = Ys[idx];
        phi_half[colbase * N + idx] = ph;
        Xs[idx] = sigma_s[(size_t)g * N + l] * (ph - phi[colbase * N + idx]);
    }
    __syncthreads();
    block_contract(Xs, N, MT, N, ncols, Ys, N);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * N; idx += blockDim.x) {
        const int cl = idx / N, n = idx - cl * N;
        const T w = (T)(h[g0 + cl] / 6.0);
        const T r0 = Ys[(2 * cl) * N + n], r1 = Ys[(2 * cl + 1) * N + n];
        rhs[(colbase + 2 * cl) * N + n] = w * (T(2) * r0 + r1);
        rhs[(colbase + 2 * cl + 1) * N + n] = w * (r0 + T(2) * r1);
    }
}

// Order-preserving key of a non-negative double (NaN sorts above +Inf).
static __device__ __forceinline__ unsigned long long dkey(double x) {
    return (unsigned long long)__double_as_longlong(fabs(x));
}

// phi_new = (phi_base ? phi_base : 0) + D v ; convergence maxima (if conv); then
// q = M (sigma_s phi_new + Q) + q_ang for the next sweep (Q, q_ang nullable).
//   SI:   phi_base = NULL, v = psi (Eq. trsi)
//   FPSA: phi_base = phi_half, v = FP correction upsilon (Eq. correct)
// conv[(r*B + b)*2 + 0] = max |phi_0 new - old|, [..+1] = max |phi_0 new|.
template <typename T>
__global__ void k_update_scatter(const T *__restrict__ v, const T *__restrict__ phi_base, T *__restrict__ phi,
                                 const T *__restrict__ sigma_s, const T *__restrict__ Qext,
                                 const T *__restrict__ DT, const T *__restrict__ MT, T *__restrict__ q,
                                 const int32_t *__restrict__ cell_inst, int B,
                                 unsigned long long *__restrict__ conv, int N, int sumK,
                                 const T *__restrict__ Qang = nullptr) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    T *Ys = Xs + 2 * kContractCells * N;
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncell = min(kContractCells, sumK - g0);
    const int ncols = 2 * ncell;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) Xs[idx] = v[colbase * N + idx];
    __syncthreads();
    block_contract(Xs, N, DT, N, ncols, Ys, N);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        const int g = g0 + c / 2;
        const size_t e = colbase * N + idx;
        T pn = Ys[idx];
        if (phi_base) pn += phi_base[e];
        if (l == 0 && conv) {
            const int slot = (r * B + cell_inst[g]) * 2;
            atomicMax(conv + slot, dkey((double)pn - (double)phi[e]));
            atomicMax(conv + slot + 1, dkey((double)pn));
        }
        phi[e] = pn;
        Xs[idx] = sigma_s[(size_t)g * N + l] * pn + (Qext ? Qext[e] : T(0));
    }
    __syncthreads();
    block_contract(Xs, N, MT, N, ncols, q + colbase * N, N, Qang ? Qang + colbase * N : nullptr);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 iterative refinement around FP32 FPSA inner solves.
// Residual of the discrete transport system (L_h - S_h) psi = m q (Eq. trop in
// LD form), in the nodal form the sweep consumes, per cell and ordinate:
//   dq = s - sigma_t psi - m^{-1} (G(mu) psi - |mu| psi_in e_up),
//   s  = M (Sigma phi + Q),  phi = D psi,
// so that the correction equation is L dpsi = S dpsi + dq with vacuum inflow
// (the source is q = M Q + q_ang; either part may be NULL).
// Also: phi (FP64) is stored and its l = 0 change against the previous outer
// iterate is max-reduced into conv (Eq. iterate on the refined iterates).
// ---------------------------------------------------------------------------
static __global__ void k_mixed_residual(const double *__restrict__ psi, double *__restrict__ phi,
                                 const double *__restrict__ sigma_s, const double *__restrict__ Qext,
                                 const double *__restrict__ DT, const double *__restrict__ MT,
                                 const double *__restrict__ sigma_t, const double *__restrict__ h,
                                 const double *__restrict__ mu, const int32_t *__restrict__ cell_inst,
                                 const int32_t *__restrict__ off, const int32_t *__restrict__ Kc, int B,
                                 unsigned long long *__restrict__ conv, float *__restrict__ dq, int N, int sumK,
                                 const double *__restrict__ Qang, const double *__restrict__ psi_inc,
                                 const int32_t *__restrict__ bc, float *__restrict__ q32,
                                 float *__restrict__ phi32) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    extern __shared__ unsigned char smem_raw[];
    double *Xs = reinterpret_cast<double *>(smem_raw);
    double *Ys = Xs + 2 * kContractCells * N;
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncell = min(kContractCells, sumK - g0);
    const int ncols = 2 * ncell;
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    const double *psr = psi + (size_t)r * sumK * 2 * N;  // this rhs
    // Both contractions use the mirror symmetry of the S_N set (mu_{N-1-n} = -mu_n,
    // equal weights, P_l(-mu) = (-1)^l P_l(mu), exact in the tables): half the FP64
    // multiply-adds of the plain products, same values up to rounding order.
    //   phi_l = sum_{n < N/2} D[l][n] (psi_n + (-1)^l psi_{N-1-n})
    //   q_n, q_{N-1-n} = E_n +- O_n,  E_n / O_n = sum over even / odd l of M[n][l] x_l
    const int h2 = N / 2;
    for (int idx = threadIdx.x; idx < ncols * h2; idx += blockDim.x) {
        const int c = idx / h2, n = idx - c * h2;
        const double a = psi[(colbase + c) * N + n], bm = psi[(colbase + c) * N + (N - 1 - n)];
        Ys[c * N + n] = a + bm;        // even part
        Ys[c * N + h2 + n] = a - bm;   // odd part
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        const double *f = Ys + c * N + ((l & 1) ? h2 : 0);
        double acc = 0.0;
#pragma unroll 8
        for (int n = 0; n < h2; ++n) acc = fma(DT[(size_t)n * N + l], f[n], acc);
        Xs[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) {
        const int c = idx / N, l = idx - c * N;
        const int g = g0 + c / 2;
        const size_t e = colbase * N + idx;
        const double pn = Xs[idx];
        if (l == 0) {
            const int slot = (r * B + cell_inst[g]) * 2;
            atomicMax(conv + slot, dkey(pn - phi[e]));
            atomicMax(conv + slot + 1, dkey(pn));
        }
        phi[e] = pn;
        Xs[idx] = sigma_s[(size_t)g * N + l] * pn + (Qext ? Qext[e] : 0.0);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncols * h2; idx += blockDim.x) {
        const int c = idx / h2, n = idx - c * h2;
        const double *x = Xs + c * N;
        double ev = 0.0, od = 0.0;
#pragma unroll 4
        for (int l = 0; l + 1 < N; l += 2) {
            ev = fma(MT[(size_t)l * N + n], x[l], ev);
            od = fma(MT[(size_t)(l + 1) * N + n], x[l + 1], od);
        }
        const double *qa = Qang ? Qang + (colbase + c) * N : nullptr;
        Ys[c * N + n] = ev + od + (qa ? qa[n] : 0.0);
        Ys[c * N + (N - 1 - n)] = ev - od + (qa ? qa[N - 1 - n] : 0.0);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncell * N; idx += blockDim.x) {
        const int cl = idx / N, n = idx - cl * N;
        const int g = g0 + cl;
        const int b = cell_inst[g], loc = g - off[b];
        const double m = mu[n], hh = h[g], st = sigma_t[g];
        const double pL = psr[((size_t)2 * g) * N + n], pR = psr[((size_t)2 * g + 1) * N + n];
        double tL, tR;
        // inflow: the upwind neighbour's outflow, else the edge value (given incoming
        // flux, or the mirror ordinate's outflow at a reflective edge)
        if (m > 0.0) {
            double pin;
            if (loc > 0) pin = psr[((size_t)2 * (g - 1) + 1) * N + n];
            else if (bc && bc[2 * b] == kBcReflect) pin = psr[((size_t)2 * g) * N + (N - 1 - n)];
            else pin = psi_inc ? psi_inc[(((size_t)r * B + b) * 2) * N + n] : 0.0;
            tL = 0.5 * m * (pL + pR) - m * pin;
            tR = 0.5 * m * (pR - pL);
        } else {
            double pin;
            if (loc < Kc[b] - 1) pin = psr[((size_t)2 * (g + 1)) * N + n];
            else if (bc && bc[2 * b + 1] == kBcReflect) pin = psr[((size_t)2 * g + 1) * N + (N - 1 - n)];
            else pin = psi_inc ? psi_inc[(((size_t)r * B + b) * 2 + 1) * N + n] : 0.0;
            tL = 0.5 * m * (pR - pL);
            tR = -0.5 * m * (pL + pR) + m * pin;  // -|mu| psi_in with mu < 0
        }
        const double w = 2.0 / hh;
        const double sL = Ys[(2 * cl) * N + n], sR = Ys[(2 * cl + 1) * N + n];
        const size_t eL = (colbase + 2 * cl) * N + n, eR = eL + N;
        const float vL = (float)(sL - st * pL - w * (2.0 * tL - tR)), vR = (float)(sR - st * pR - w * (2.0 * tR - tL));
        dq[eL] = vL;
        dq[eR] = vR;
        // the inner FP32 solve starts from zero moments with this source (q32, phi32 NULL: not wanted)
        if (q32) {
            q32[eL] = vL;
            q32[eR] = vR;
        }
        if (phi32) {
            phi32[eL] = 0.f;
            phi32[eR] = 0.f;
        }
    }
}

// psi64 += dpsi, dpsi = psi_half + upsilon of the last inner FPSA iteration (Eq. correct);
// ups NULL: dpsi = psi_half (inner SI, or the sweep after an inner GMRES solve).
static __global__ void k_mixed_accumulate(double *__restrict__ psi, const float *__restrict__ psi_half,
                                   const float *__restrict__ ups, size_t n) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        psi[i] += (double)psi_half[i] + (ups ? (double)ups[i] : 0.0);
}

// x (moments, padded to N) -> nodal angular values M x, used to turn a moment
// initial guess into an angular one.
template <typename T>
__global__ void k_expand(const T *__restrict__ x, const T *__restrict__ MT, T *__restrict__ out, int N, int sumK) {
    extern __shared__ unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    const int r = blockIdx.y;
    const int g0 = blockIdx.x * kContractCells;
    const int ncols = 2 * min(kContractCells, sumK - g0);
    const size_t colbase = ((size_t)r * sumK + g0) * 2;
    for (int idx = threadIdx.x; idx < ncols * N; idx += blockDim.x) Xs[idx] = x[colbase * N + idx];
    __syncthreads();
    block_contract(Xs, N, MT, N, ncols, out + colbase * N, N);
}

// Worst relative change over (rhs, instance); resets the accumulators.
// out[0] = max_rb conv_d / conv_a (NaN if any value was non-finite).
static __global__ void k_conv_finalize(unsigned long long *conv, int nrb, double *out) {
    tc::grid_dependency_wait();  // inputs of the previous kernel (programmatic dependent launch)
    __shared__ double red[256];
    double worst = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < nrb; i += blockDim.x) {
        double d = __longlong_as_double((long long)conv[2 * i]);
        double a = __longlong_as_double((long long)conv[2 * i + 1]);
        if (!isfinite(d) || !isfinite(a)) bad = true;
        double e = (a > 0.0) ? d / a : (d > 0.0 ? INFINITY : 0.0);
        worst = fmax(worst, e);
        conv[2 * i] = 0ull;
        conv[2 * i + 1] = 0ull;
    }
    red[threadIdx.x] = bad ? NAN : worst;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double x = red[threadIdx.x], y = red[threadIdx.x + s];
            red[threadIdx.x] = (isnan(x) || isnan(y)) ? NAN : fmax(x, y);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// ---------------------------------------------------------------------------
// Cross sections and sources of fpsa_set_xs, converted on the device from the
// caller's FP64 layout (moments l < L+1) to the padded working layouts (l < N):
// sigma_s -> sig64 / sig32 [sumK][N], q -> Q64 / Q32 [R][sumK][2][N] (any output
// may be NULL), sigma_t, sigma_s0, sigma_s1 per cell. Validation (the first failing
// cell wins, in the order sigma_t, finite sigma_s, 0 <= sigma_s0 <= sigma_t):
// *err_cell = min(4 cell + check), *err_q = 1 on a non-finite source moment.
// ---------------------------------------------------------------------------
static __global__ void k_prepare_xs(const double *__restrict__ st_in, const double *__restrict__ ss_in,
                                    const double *__restrict__ q_in, int N, int L1, int sumK, int R,
                                    double *__restrict__ sig64, float *__restrict__ sig32, double *__restrict__ Q64,
                                    float *__restrict__ Q32, double *__restrict__ d_st, double *__restrict__ d_s0,
                                    double *__restrict__ d_s1, int *__restrict__ err_cell, int *__restrict__ err_q) {
    const size_t nthr = (size_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (size_t c = t0; c < (size_t)sumK; c += nthr) {
        const double st = st_in[c], s0 = ss_in[c * L1], s1 = L1 > 1 ? ss_in[c * L1 + 1] : 0.0;
        int check = -1;
        if (!isfinite(st) || !(st > 0.0)) check = 0;
        else {
            for (int l = 0; l < L1 && check < 0; ++l)
                if (!isfinite(ss_in[c * L1 + l])) check = 1;
            if (check < 0 && (s0 < 0.0 || s0 > st)) check = 2;
        }
        if (check >= 0) atomicMin(err_cell, (int)(4 * c) + check);
        d_st[c] = st;
        d_s0[c] = s0;
        d_s1[c] = s1;
    }
    for (size_t e = t0; e < (size_t)sumK * N; e += nthr) {
        const size_t c = e / N;
        const int l = (int)(e - c * N);
        const double v = l < L1 ? ss_in[c * L1 + l] : 0.0;
        if (sig64) sig64[e] = v;
        if (sig32) sig32[e] = (float)v;
    }
    const size_t ncol = (size_t)R * sumK * 2;
    for (size_t e = t0; e < ncol * N; e += nthr) {
        const size_t col = e / N;
        const int l = (int)(e - col * N);
        const double v = l < L1 ? q_in[col * L1 + l] : 0.0;
        if (!isfinite(v)) *err_q = 1;
        if (Q64) Q64[e] = v;
        if (Q32) Q32[e] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// FP operator, LD in space (Eqs. fpop, fp-mpd-oper, wd-eq-oper):
//   mu d/dz + K_g,  K_g = sigma_a I - sigma_tr/2 A_FP,
// cell block A_g[a*N+n][b*N+m] = G(mu_n)_ab delta_nm + m_ab K_g[n][m] with
// G(mu) = [[mu/2 - mu[mu<0], mu/2], [-mu/2, -mu/2 + mu[mu>0]]], m = (h/6)[[2,1],[1,2]].
// Upwind couplings at level 0: B_g[p][p] = -mu_{N/2+p} (row L+ of g, column
// R+ of g-1), C_g[p][p] = mu_p (row R- of g, column L- of g+1).
// ---------------------------------------------------------------------------
// Arithmetic in T (per-cell scalars in FP64, rounded once; mu passed in T): FP64
// throughput is a small fraction of FP32 on this GPU, and the FP32 factor path
// stores T anyway. Block (32, 8): x runs over the 2N columns of a row (coalesced
// stores), y over rows. Reflective edges add -|mu_n| at (incoming n, mirror N-1-n)
// of the edge node.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fp_assemble(const T *__restrict__ muT, const T *__restrict__ Afp,
                              const double *__restrict__ h, const double *__restrict__ sigma_t,
                              const double *__restrict__ sigma_s0, const double *__restrict__ sigma_s1,
                              const int32_t *__restrict__ cell_inst, const int32_t *__restrict__ off,
                              const int32_t *__restrict__ Kc, const int32_t *__restrict__ slot_base, int N,
                              T *__restrict__ A, T *__restrict__ Bc, T *__restrict__ Cc,
                              const int32_t *__restrict__ bc = nullptr) {
    const int g = blockIdx.x;
    const int b = cell_inst[g];
    const int local = g - off[b];
    const bool refl_l = bc && local == 0 && bc[2 * b] == kBcReflect;
    const bool refl_r = bc && local == Kc[b] - 1 && bc[2 * b + 1] == kBcReflect;
    const int n2 = 2 * N, h2 = N / 2;
    // the cell's scalars, formed once per block in FP64 (kept in shared memory so the
    // compiler does not re-form the FP64 divisions inside the element loop)
    __shared__ T sc[4];
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const double hh = h[g];
        sc[0] = (T)(hh / 3.0);
        sc[1] = (T)(hh / 6.0);
        sc[2] = (T)(sigma_t[g] - sigma_s0[g]);
        sc[3] = (T)(-0.5 * (sigma_s0[g] - sigma_s1[g]));
    }
    __syncthreads();
    const T m_d = sc[0], m_o = sc[1], sa = sc[2], hs = sc[3];
    T *Ag = A + (size_t)g * n2 * n2;
    for (int row = threadIdx.y; row < n2; row += blockDim.y) {
        const int a = row >= N, n = row - a * N;
        const T x = muT[n], half = T(0.5) * x;
        const T gdiag = (a == 0) ? (x > T(0) ? half : -half) : (x > T(0) ? half : -half);  // G_aa
        const T goff = (a == 0) ? half : -half;                                               // G_a,1-a
        const bool refl = (refl_l && a == 0 && x > T(0)) || (refl_r && a == 1 && x < T(0));
        const T* arow = Afp + (size_t)n * N;
        T *out = Ag + (size_t)row * n2;
        for (int col = threadIdx.x; col < n2; col += blockDim.x) {
            const int bb = col >= N, m = col - bb * N;
            T v = (a == bb ? m_d : m_o) * fma(hs, arow[m], n == m ? sa : T(0));
            if (n == m) v += (a == bb) ? gdiag : goff;
            if (refl && a == bb && m == N - 1 - n) v -= (x > T(0) ? x : -x);
            out[col] = v;
        }
    }
    T *Bg = Bc + (size_t)slot_base[g] * h2 * h2;
    T *Cg = Cc + (size_t)slot_base[g] * h2 * h2;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int idx = tid; idx < h2 * h2; idx += nt) {
        const int p = idx / h2, qq = idx - p * h2;
        Bg[idx] = (p == qq && local > 0) ? -muT[h2 + p] : T(0);
        Cg[idx] = (p == qq && local < Kc[b] - 1) ? muT[p] : T(0);
    }
}

// ---------------------------------------------------------------------------
// Block cyclic reduction, factorization. Gauss-Jordan inversion with partial
// pivoting of the eliminated cells' 2N x 2N blocks, in shared memory; the
// inverse is written back transposed. Growth check (always in FP64):
// max|A| * max|A^{-1}| per block, max-reduced into *growth; a zero or
// non-finite pivot sets *status = 1.
// ---------------------------------------------------------------------------
// Body shared by the in-place kernel below and the strided sub-block variant:
// src / dst are n2 x n2 row-major with leading dimensions lds / ldd (they may be
// the same memory); the inverse is written transposed (dst[c][r]) when tout.
// growth may be NULL (no growth report).
template <typename T>
__device__ __forceinline__ void gj_smem_body(const T *src, int lds, T *dst, int ldd, bool tout, int n2,
                                             unsigned long long *__restrict__ growth, int *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    const int ld = n2 + 1;
    T *a = reinterpret_cast<T *>(smem_raw);
    T *colk = a + (size_t)n2 * ld;
    int *perm = reinterpret_cast<int *>(colk + n2);
    __shared__ double s_amax;
    __shared__ int s_piv;
    __shared__ T s_pval;
    double amax = 0.0;
    for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
        const int i = idx / n2, j = idx - i * n2;
        const T v = __ldcg(src + (size_t)i * lds + j);
        a[i * ld + j] = v;
        amax = fmax(amax, fabs((double)v));
    }
    // block max of |A|
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (threadIdx.x == 0) s_amax = 0.0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&s_amax, dkey(amax));
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < n2; ++k) {
        // pivot search in column k, rows k..n2-1 (warp 0)
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + threadIdx.x; i < n2; i += 32) {
                const double v = fabs((double)a[i * ld + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) { s_piv = bi; perm[k] = bi; }
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k)
            for (int j = threadIdx.x; j < n2; j += blockDim.x) {
                const T t = a[k * ld + j];
                a[k * ld + j] = a[p * ld + j];
                a[p * ld + j] = t;
            }
        __syncthreads();
        if (threadIdx.x == 0) s_pval = a[k * ld + k];
        for (int i = threadIdx.x; i < n2; i += blockDim.x) colk[i] = a[i * ld + k];
        __syncthreads();
        const T pv = s_pval;
        if (pv == T(0) || !isfinite((double)pv)) bad = true;
        const T inv = T(1) / pv;
        // scale pivot row; column k of the pivot row becomes 1/pv
        for (int j = threadIdx.x; j < n2; j += blockDim.x) a[k * ld + j] = (j == k) ? inv : a[k * ld + j] * inv;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
            const int i = idx / n2, j = idx - i * n2;
            if (i == k) continue;
            const T f = colk[i];
            if (j == k) a[i * ld + j] = -f * inv;
            else a[i * ld + j] = fma(-f, a[k * ld + j], a[i * ld + j]);
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = n2 - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k)
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const T t = a[i * ld + k];
                a[i * ld + k] = a[i * ld + p];
                a[i * ld + p] = t;
            }
        __syncthreads();
    }
    double ainv = 0.0;
    for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
        const int c = idx / n2, rr = idx - c * n2;  // inv[rr][c]
        const T v = a[rr * ld + c];
        if (tout) dst[(size_t)c * ldd + rr] = v;
        else dst[(size_t)rr * ldd + c] = v;
        ainv = fmax(ainv, fabs((double)v));
        if (!isfinite((double)v)) bad = true;
    }
    for (int o = 16; o > 0; o >>= 1) ainv = fmax(ainv, __shfl_xor_sync(0xffffffffu, ainv, o));
    if (growth && (threadIdx.x & 31) == 0) atomicMax(growth, dkey(ainv * s_amax));
    if (bad) atomicExch(status, 1);
}

// In place, inverse written back transposed (the layout the BCR solve reads).
template <typename T>
__global__ void k_bcr_invert(T *__restrict__ A, const BcrItem *__restrict__ items, int n2,
                             unsigned long long *__restrict__ growth, int *__restrict__ status) {
    T *Ag = A + (size_t)items[blockIdx.x].cell * n2 * n2;
    gj_smem_body(Ag, n2, Ag, n2, true, n2, growth, status);
}

// Register-tiled Gauss-Jordan inversion for n2 = 2N in {32, 64, 128}: 16 warps;
// warp w owns the columns w + 16 j (j < n2/16), lane t the rows t + 32 i
// (i < n2/32), so every thread holds an (n2/32) x (n2/16) tile in registers and
// column k lives in one warp. Pivoting is implicit: step k picks, among rows not
// yet used, the row p_k of largest |a[p][k]| (partial pivoting without moving
// rows; the comparison key is |a| rounded to FP32). The in-place update is the
// usual one with row p_k as pivot row; at the end the array X holds
// A^{-1}[r][c] = X[p_r][q_c] with q the inverse of p (row p_k carries step k's
// identity column). Written back transposed.
//
// One block barrier per step: the pivot row reaches the other lanes of each warp
// by shuffles (every warp holds all rows of its columns), only column k goes
// through shared memory, and the warp owning column k+1 updates that column first
// and picks pivot k+1 (look-ahead) while the other warps are still updating.
// Body shared by the in-place kernel and the strided sub-block variant: src / dst
// are N2 x N2 row-major with leading dimensions lds / ldd; transposed output when
// tout; growth may be NULL.
template <typename T, int RI>
__device__ __forceinline__ void gj_pick_pivot(const T (&colv)[RI], unsigned used, int lane, int &p) {
    // key 0: no candidate; else the FP32 bits of |v| plus one (|v| >= 0 orders as unsigned)
    unsigned best = 0u;
    int bi = 0;
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        const unsigned key = (used >> i) & 1u ? 0u : __float_as_uint(fabsf((float)colv[i])) + 1u;
        if (key > best) { best = key; bi = lane + 32 * i; }
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, best);
    const unsigned who = __ballot_sync(0xffffffffu, best == m);
    p = __shfl_sync(0xffffffffu, bi, __ffs(who) - 1);
}

// rv[j] = (row ip of lane pl's register tile)[j] * inv, broadcast to the warp by
// shuffles; ip and pl are warp-uniform, so the row is chosen by a branch.
template <typename T, int RI, int CJ>
__device__ __forceinline__ void gj_pivot_row(const T (&x)[RI][CJ], int ip, int pl, T inv, T (&rv)[CJ]) {
#pragma unroll
    for (int i = 0; i < RI; ++i)
        if (i == ip) {
#pragma unroll
            for (int j = 0; j < CJ; ++j) rv[j] = __shfl_sync(0xffffffffu, x[i][j], pl) * inv;
        }
}

// x[I][j] = rv[j] for every j except jskip (the look-ahead column, already set).
template <typename T, int RI, int CJ, int I>
__device__ __forceinline__ void gj_set_row_i(T (&x)[RI][CJ], const T (&rv)[CJ], int jskip) {
    if constexpr (I < RI) {
#pragma unroll
        for (int j = 0; j < CJ; ++j)
            if (j != jskip) x[I][j] = rv[j];
    }
}

template <typename T, int RI, int CJ>
__device__ __forceinline__ void gj_set_row_elem(T (&x)[RI][CJ], int ip, int j, T val) {
#pragma unroll
    for (int i = 0; i < RI; ++i)
        if (i == ip) x[i][j] = val;
}

template <typename T, int N2>
struct GjShared {
    T (*colbuf)[N2];
    int *s_p, *perm, *iperm;
};

// One elimination step k = 16 JK + wk with the look-ahead column register JN
// (JN = CJ: no look-ahead, the last step).
template <typename T, int N2, int JK, int JN>
__device__ __forceinline__ void gj_step(T (&x)[N2 / 32][N2 / 16], const GjShared<T, N2> &sh, unsigned &used,
                                        bool &bad, int lane, int w, int wk) {
    constexpr int RI = N2 / 32, CJ = N2 / 16;
    const int k = 16 * JK + wk, b = k & 1;
    const int p = sh.s_p[b];
    const T pv = sh.colbuf[b][p];
    if (pv == T(0) || !isfinite(pv)) bad = true;
    const T inv = __frcp_rn(pv);  // correctly rounded, as 1 / pv
    const int ip = p >> 5, pl = p & 31;
    if (lane == pl) used |= 1u << ip;
    T f[RI], rv[CJ];
#pragma unroll
    for (int i = 0; i < RI; ++i) f[i] = sh.colbuf[b][lane + 32 * i];
    gj_pivot_row<T, RI, CJ>(x, ip, pl, inv, rv);  // pivot row of this warp's columns, from lane pl
    if (w == wk) {  // column k: its old value is replaced, not updated
        rv[JK] = inv;
#pragma unroll
        for (int i = 0; i < RI; ++i) x[i][JK] = T(0);
    }
    bool ahead = false;
    if constexpr (JN < CJ) {
        ahead = w == ((wk + 1) & 15);
        if (ahead) {
            // look-ahead: update column k+1 now and pick pivot k+1
            T colv[RI];
#pragma unroll
            for (int i = 0; i < RI; ++i) x[i][JN] = fma(-f[i], rv[JN], x[i][JN]);
            if (lane == pl) gj_set_row_elem<T, RI, CJ>(x, ip, JN, rv[JN]);
#pragma unroll
            for (int i = 0; i < RI; ++i) {
                colv[i] = x[i][JN];
                sh.colbuf[b ^ 1][lane + 32 * i] = colv[i];
            }
            int pn;
            gj_pick_pivot<T, RI>(colv, used, lane, pn);
            if (lane == 0) {
                sh.s_p[b ^ 1] = pn;
                sh.perm[k + 1] = pn;
                sh.iperm[pn] = k + 1;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
        if (j == JN && ahead) continue;
#pragma unroll
        for (int i = 0; i < RI; ++i) x[i][j] = fma(-f[i], rv[j], x[i][j]);
    }
    // the pivot row becomes the scaled row (its own update used f = pv)
    if (lane == pl) {
        const int js = ahead ? JN : -1;
        switch (ip) {
            case 0: gj_set_row_i<T, RI, CJ, 0>(x, rv, js); break;
            case 1: gj_set_row_i<T, RI, CJ, 1>(x, rv, js); break;
            case 2: gj_set_row_i<T, RI, CJ, 2>(x, rv, js); break;
            default: gj_set_row_i<T, RI, CJ, 3>(x, rv, js); break;
        }
    }
    __syncthreads();
}

// All steps with column register JK (k = 16 JK .. 16 JK + 15), then JK + 1.
template <typename T, int N2, int JK>
__device__ __forceinline__ void gj_steps(T (&x)[N2 / 32][N2 / 16], const GjShared<T, N2> &sh, unsigned &used,
                                         bool &bad, int lane, int w) {
    constexpr int CJ = N2 / 16;
    if constexpr (JK < CJ) {
        for (int wk = 0; wk < 15; ++wk) gj_step<T, N2, JK, JK>(x, sh, used, bad, lane, w, wk);
        gj_step<T, N2, JK, JK + 1>(x, sh, used, bad, lane, w, 15);
        gj_steps<T, N2, JK + 1>(x, sh, used, bad, lane, w);
    }
}

// One row of CJ values to / from shared memory in 16-byte (CJ % 4 == 0) or 8-byte vectors.
template <int CJ>
__device__ __forceinline__ void gj_st_row(float *d, const float (&v)[CJ]) {
    if constexpr (CJ % 4 == 0) {
#pragma unroll
        for (int j = 0; j < CJ; j += 4) *reinterpret_cast<float4 *>(d + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < CJ; j += 2) *reinterpret_cast<float2 *>(d + j) = make_float2(v[j], v[j + 1]);
    }
}
template <int CJ>
__device__ __forceinline__ void gj_ld_row(float (&v)[CJ], const float *s) {
    if constexpr (CJ % 4 == 0) {
#pragma unroll
        for (int j = 0; j < CJ; j += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(s + j);
            v[j] = t.x; v[j + 1] = t.y; v[j + 2] = t.z; v[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < CJ; j += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(s + j);
            v[j] = t.x; v[j + 1] = t.y;
        }
    }
}

// Blocked Gauss-Jordan inversion (FP32) for n2 = N2 in {32, 64, 128}: 16 warps, warp
// w owns the CJ = N2/16 consecutive columns CJ w .. CJ w + CJ - 1 (a panel), lane t
// the rows t + 32 i. Panel q is eliminated by its owner warp alone (CJ pivot steps
// with partial pivoting: one warp max reduction per step, whose key carries the
// magnitude to 16 mantissa bits and the row index in its low 7 bits, and shuffles of
// the pivot row), which leaves in its columns W = E[:, P], E the product of the
// panel's elementary transformations and P its pivot rows; every other warp then
// applies E to its own columns,
//   X[r][c] <- (r in P ? 0 : X[r][c]) + sum_j W[r][j] X[P_j][c],
// a rank-CJ update (the lanes holding a pivot row publish this warp's part of it, PR,
// before it restarts from 0). One block barrier per panel (16 in all); the owner of
// panel q+1 starts eliminating as soon as its own update for panel q is done. The
// result is the in-place inverse of the unblocked elimination with the same pivots
// (only the rounding order of the updates differs): A^{-1}[r][c] = X[p_r][q_c].
// The reciprocal of the pivot is rcp.approx refined by one Newton step.
template <int N2>
__device__ __forceinline__ void gj_panel_body(const float *src, int lds, float *dst, int ldd, bool tout,
                                              unsigned long long *__restrict__ growth, int *__restrict__ status) {
    static_assert(N2 >= 32 && N2 <= 128 && N2 % 32 == 0, "row index must fit the 7 key bits");
    constexpr int RI = N2 / 32, CJ = N2 / 16;
    constexpr int WS = (CJ % 4 == 0) ? CJ + 4 : CJ;  // padded W row: conflict-free 16-byte accesses
    __shared__ __align__(16) float Wb[2][N2][WS];
    __shared__ __align__(16) float PRb[16][CJ][CJ];
    __shared__ int piv_panel[N2], perm[N2], iperm[N2];
    __shared__ double s_red[16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float x[RI][CJ];
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        // this lane's CJ consecutive values of row lane + 32 i (16-byte / 8-byte vectors)
        const float *rp = src + (size_t)(lane + 32 * i) * lds + CJ * w;
        if constexpr (CJ % 4 == 0) {
#pragma unroll
            for (int j = 0; j < CJ; j += 4) {
                const float4 v = __ldcg(reinterpret_cast<const float4 *>(rp + j));
                x[i][j] = v.x; x[i][j + 1] = v.y; x[i][j + 2] = v.z; x[i][j + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < CJ; j += 2) {
                const float2 v = __ldcg(reinterpret_cast<const float2 *>(rp + j));
                x[i][j] = v.x; x[i][j + 1] = v.y;
            }
        }
#pragma unroll
        for (int j = 0; j < CJ; ++j) amax = fmaxf(amax, fabsf(x[i][j]));
    }
    for (int r = threadIdx.x; r < N2; r += blockDim.x) piv_panel[r] = -1;
    unsigned used = 0u;  // bit i: row lane + 32 i has been a pivot row
    bool bad = false;
    __syncthreads();
    for (int q = 0; q < 16; ++q) {
        const int qb = q & 1;
        if (w == q) {
#pragma unroll
            for (int c = 0; c < CJ; ++c) {
                float colv[RI];
#pragma unroll
                for (int i = 0; i < RI; ++i) colv[i] = x[i][c];
                // pivot: the largest |value| among the rows not yet used, its row index in
                // the low 7 bits of the key (magnitudes compared to 16 mantissa bits; ties
                // go to the larger row): one warp max reduction gives the row
                unsigned best = 0u;
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const unsigned mag = (__float_as_uint(colv[i]) & 0x7fffffffu) >> 7;
                    const unsigned key = ((used >> i) & 1u) ? 0u : (((mag + 1u) << 7) | unsigned(lane + 32 * i));
                    best = max(best, key);
                }
                const int p = int(__reduce_max_sync(0xffffffffu, best) & 127u);
                const int ip = p >> 5, pl = p & 31;
                // pivot row of this warp's columns (select chain on the warp-uniform ip)
                float rv[CJ];
#pragma unroll
                for (int j = 0; j < CJ; ++j) {
                    float v = x[0][j];
#pragma unroll
                    for (int i = 1; i < RI; ++i) v = (ip == i) ? x[i][j] : v;
                    rv[j] = __shfl_sync(0xffffffffu, v, pl);
                }
                const float pv = rv[c];
                if (pv == 0.f || !isfinite(pv)) bad = true;
                float inv;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(pv));
                inv = inv * fmaf(-pv, inv, 2.f);  // one Newton step for 1/pv
#pragma unroll
                for (int j = 0; j < CJ; ++j) rv[j] = (j == c) ? inv : rv[j] * inv;
                // x <- s_i x + g_i rv: s = 1, g = -x[i][c] for the other rows (column c
                // first cleared: it is replaced), s = 0, g = 1 for the pivot row
                float sg[RI], gg[RI];
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const bool prow = lane == pl && i == ip;
                    sg[i] = prow ? 0.f : 1.f;
                    gg[i] = prow ? 1.f : -x[i][c];
                    x[i][c] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < RI; ++i)
#pragma unroll
                    for (int j = 0; j < CJ; j += 2) {
                        float2 xv = make_float2(x[i][j], x[i][j + 1]);
                        xv = __ffma2_rn(make_float2(gg[i], gg[i]), make_float2(rv[j], rv[j + 1]),
                                        __fmul2_rn(make_float2(sg[i], sg[i]), xv));
                        x[i][j] = xv.x;
                        x[i][j + 1] = xv.y;
                    }
                used |= (lane == pl) ? (1u << ip) : 0u;
                if (lane == 0) {
                    const int k = q * CJ + c;
                    perm[k] = p;
                    iperm[p] = k;
                    piv_panel[p] = q;
                }
            }
#pragma unroll
            for (int i = 0; i < RI; ++i) gj_st_row<CJ>(&Wb[qb][lane + 32 * i][0], x[i]);
        }
        __syncthreads();
        if (w != q) {
            // this warp's values of the panel's pivot rows -> PRb[w] (old values), then those
            // rows restart from 0: X[r][:] <- (r in P ? 0 : X[r][:]) + W[r][:] PR
#pragma unroll
            for (int i = 0; i < RI; ++i) {
                const int row = lane + 32 * i;
                if (piv_panel[row] == q) {
                    gj_st_row<CJ>(&PRb[w][iperm[row] - q * CJ][0], x[i]);
                    used |= 1u << i;
#pragma unroll
                    for (int j = 0; j < CJ; ++j) x[i][j] = 0.f;
                }
            }
            __syncwarp();
            // two W columns at a time: 8-byte W loads per row, two pivot rows of PR
#pragma unroll
            for (int c = 0; c < CJ; c += 2) {
                float prc[2][CJ];
                gj_ld_row<CJ>(prc[0], &PRb[w][c][0]);
                gj_ld_row<CJ>(prc[1], &PRb[w][c + 1][0]);
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const float2 wv = *reinterpret_cast<const float2 *>(&Wb[qb][lane + 32 * i][c]);
#pragma unroll
                    for (int j = 0; j < CJ; j += 2) {
                        float2 acc = make_float2(x[i][j], x[i][j + 1]);
                        acc = __ffma2_rn(make_float2(wv.x, wv.x), make_float2(prc[0][j], prc[0][j + 1]), acc);
                        acc = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(prc[1][j], prc[1][j + 1]), acc);
                        x[i][j] = acc.x;
                        x[i][j + 1] = acc.y;
                    }
                }
            }
        }
    }
    __syncthreads();
    // X[row][col] = A^{-1}[r][c] with r = iperm[row], c = perm[col]; written transposed when tout
    float ainv = 0.f;
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
            const int row = lane + 32 * i, col = CJ * w + j;
            const int r = iperm[row], c = perm[col];
            if (tout) dst[(size_t)c * ldd + r] = x[i][j];
            else dst[(size_t)r * ldd + c] = x[i][j];
            ainv = fmaxf(ainv, fabsf(x[i][j]));
            if (!isfinite(x[i][j])) bad = true;
        }
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        ainv = fmaxf(ainv, __shfl_xor_sync(0xffffffffu, ainv, o));
    }
    if (lane == 0) s_red[w] = (double)amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < 16; ++i) m = fmax(m, s_red[i]);
        s_red[0] = m;
    }
    __syncthreads();
    if (growth && lane == 0) atomicMax(growth, dkey((double)ainv * s_red[0]));
    if (bad) atomicExch(status, 1);
}

template <typename T, int N2>
__device__ __forceinline__ void gj_reg_body(const T *src, int lds, T *dst, int ldd, bool tout,
                                            unsigned long long *__restrict__ growth, int *__restrict__ status) {
    constexpr int RI = N2 / 32, CJ = N2 / 16;
    __shared__ T colbuf[2][N2];
    __shared__ int s_p[2], perm[N2], iperm[N2];
    __shared__ double s_red[16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x[RI][CJ];
    T amax = T(0);  // growth bookkeeping in T (FP64 only for the final product)
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
            x[i][j] = __ldcg(src + (size_t)(lane + 32 * i) * lds + w + 16 * j);
            amax = fmax(amax, fabs(x[i][j]));
        }
    unsigned used = 0u;  // bit i: row lane + 32 i has been a pivot row
    bool bad = false;
    if (w == 0) {  // pivot of step 0 (column 0 = x[.][0] of warp 0)
        T colv[RI];
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            colv[i] = x[i][0];
            colbuf[0][lane + 32 * i] = colv[i];
        }
        int pn;
        gj_pick_pivot<T, RI>(colv, used, lane, pn);
        if (lane == 0) {
            s_p[0] = pn;
            perm[0] = pn;
            iperm[pn] = 0;
        }
    }
    __syncthreads();
    // step k = 16 JK + wk: column k is x[.][JK] of warp wk. JK is a compile-time index
    // (the loop over it is unrolled) so the owner's and the look-ahead column's
    // registers are addressed statically; the look-ahead column is JK (wk < 15) or
    // JK + 1 (wk = 15).
    // (FP32; the FP64 tile is register-bound, so there the loop stays rolled)
    if constexpr (sizeof(T) == 4) {
        GjShared<T, N2> sh{colbuf, s_p, perm, iperm};
        gj_steps<T, N2, 0>(x, sh, used, bad, lane, w);
    } else {
        for (int k = 0; k < N2; ++k) {
            const int b = k & 1;
            const int p = s_p[b];
            const T pv = colbuf[b][p];
            if (pv == T(0) || !isfinite(pv)) bad = true;
            const T inv = T(1) / pv;
            const int ip = p >> 5, pl = p & 31;
            if (lane == pl) used |= 1u << ip;
            T f[RI], rv[CJ];
    #pragma unroll
            for (int i = 0; i < RI; ++i) f[i] = colbuf[b][lane + 32 * i];
            // pivot row values of this warp's columns, from lane pl
            gj_pivot_row<T, RI, CJ>(x, ip, pl, inv, rv);
            const bool own = w == (k & 15);
            const int jk = k >> 4;
            if (own) {  // column k: its old value is replaced, not updated
    #pragma unroll
                for (int j = 0; j < CJ; ++j)
                    if (j == jk) {
                        rv[j] = inv;
    #pragma unroll
                        for (int i = 0; i < RI; ++i) x[i][j] = T(0);
                    }
            }
            const bool ahead = k + 1 < N2 && w == ((k + 1) & 15);
            const int jn = (k + 1) >> 4;
            if (ahead) {
                // look-ahead: update column k+1 now and pick pivot k+1
                T colv[RI];
    #pragma unroll
                for (int j = 0; j < CJ; ++j)
                    if (j == jn) {
    #pragma unroll
                        for (int i = 0; i < RI; ++i) x[i][j] = fma(-f[i], rv[j], x[i][j]);
                        if (lane == pl) gj_set_row_elem<T, RI, CJ>(x, ip, j, rv[j]);
    #pragma unroll
                        for (int i = 0; i < RI; ++i) colv[i] = x[i][j];
                    }
    #pragma unroll
                for (int i = 0; i < RI; ++i) colbuf[b ^ 1][lane + 32 * i] = colv[i];
                int pn;
                gj_pick_pivot<T, RI>(colv, used, lane, pn);
                if (lane == 0) {
                    s_p[b ^ 1] = pn;
                    perm[k + 1] = pn;
                    iperm[pn] = k + 1;
                }
            }
    #pragma unroll
            for (int j = 0; j < CJ; ++j) {
                if (ahead && j == jn) continue;
    #pragma unroll
                for (int i = 0; i < RI; ++i) x[i][j] = fma(-f[i], rv[j], x[i][j]);
            }
            // the pivot row becomes the scaled row (its own update used f = pv)
            if (lane == pl) {
                const int js = ahead ? jn : -1;
                switch (ip) {
                    case 0: gj_set_row_i<T, RI, CJ, 0>(x, rv, js); break;
                    case 1: gj_set_row_i<T, RI, CJ, 1>(x, rv, js); break;
                    case 2: gj_set_row_i<T, RI, CJ, 2>(x, rv, js); break;
                    default: gj_set_row_i<T, RI, CJ, 3>(x, rv, js); break;
                }
            }
            __syncthreads();
        }
    }
    // Thread holds X[row][col] = A^{-1}[r][c] with perm[r] = row (r = iperm[row]) and
    // iperm[c] = col (c = perm[col]); written transposed when tout.
    T ainv = T(0);
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
            const int row = lane + 32 * i, col = w + 16 * j;
            const int r = iperm[row], c = perm[col];
            if (tout) dst[(size_t)c * ldd + r] = x[i][j];
            else dst[(size_t)r * ldd + c] = x[i][j];
            ainv = fmax(ainv, fabs(x[i][j]));
            if (!isfinite(x[i][j])) bad = true;
        }
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        ainv = fmax(ainv, __shfl_xor_sync(0xffffffffu, ainv, o));
    }
    if (lane == 0) s_red[w] = (double)amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < 16; ++i) m = fmax(m, s_red[i]);
        s_red[0] = m;
    }
    __syncthreads();
    if (growth && lane == 0) atomicMax(growth, dkey((double)ainv * s_red[0]));
    if (bad) atomicExch(status, 1);
}

template <typename T>
__device__ __forceinline__ void schur_body(T *__restrict__ A, T *__restrict__ Bc, T *__restrict__ Cc,
                                           const BcrItem &it, int N, int staged, unsigned char *smem_raw);

template <typename T, int N2>
__global__ void __launch_bounds__(512) k_bcr_invert_reg(T *__restrict__ A, const BcrItem *__restrict__ items,
                                                        unsigned long long *__restrict__ growth,
                                                        int *__restrict__ status, T *__restrict__ Bc = nullptr,
                                                        T *__restrict__ Cc = nullptr, int schur_staged = -1) {
    const BcrItem it = items[blockIdx.x];
    T *Ag = A + (size_t)it.cell * N2 * N2;
    if constexpr (sizeof(T) == 4) gj_panel_body<N2>(Ag, N2, Ag, N2, true, growth, status);
    else gj_reg_body<T, N2>(Ag, N2, Ag, N2, true, growth, status);
    if (schur_staged >= 0) {
        // the level's Schur updates of this cell's neighbours, from the inverse this block
        // just wrote (block barrier: its global writes are visible to the whole block)
        extern __shared__ unsigned char smem_dyn[];
        __syncthreads();
        schur_body(A, Bc, Cc, it, N2 / 2, schur_staged, smem_dyn);
    }
}

// A load that bypasses L1 when p is in global memory (data another block may have
// written during the same launch), a plain load for shared memory.
template <typename T>
__device__ __forceinline__ T ld_fresh(const T *p) {
    return __isGlobal(p) ? __ldcg(p) : *p;
}

// out (+)= X Y for h2 x h2 operands through shared memory: both operands are
// staged with coalesced loads (the index that is contiguous in memory runs
// fastest across threads), then every thread forms a 2 x 2 register tile.
// buf holds 2 h2^2 values. mode: 0 store, 1 subtract from out, 2 store negated.
// With buf == NULL (blocks too large to stage) the operands are read from global
// memory directly, one output per thread.
template <typename T>
__device__ __forceinline__ void smem_mm(T *out, int ldo, int mode, const T *X, int xr, int xc, const T *Y, int yr,
                                        int yc, int h2, T *buf) {
    const int hh = h2 * h2;
    if (!buf) {
        for (int idx = threadIdx.x; idx < hh; idx += blockDim.x) {
            const int p = idx / h2, q = idx - p * h2;
            T acc = T(0);
            for (int kk = 0; kk < h2; ++kk)
                acc = fma(ld_fresh(X + (size_t)p * xr + (size_t)kk * xc), ld_fresh(Y + (size_t)kk * yr + (size_t)q * yc), acc);
            T *o = out + (size_t)p * ldo + q;
            if (mode == 1) *o = ld_fresh(o) - acc;
            else if (mode == 2) *o = -acc;
            else *o = acc;
        }
        __syncthreads();
        return;
    }
    T *Xs = buf, *Ys = buf + h2 * h2;  // Xs[p][k], Ys[k][q]
    for (int idx = threadIdx.x; idx < hh; idx += blockDim.x) {
        int p, kk;
        if (xr == 1) { p = idx % h2; kk = idx / h2; } else { kk = idx % h2; p = idx / h2; }
        Xs[p * h2 + kk] = ld_fresh(X + (size_t)p * xr + (size_t)kk * xc);
        int k2, q;
        if (yr == 1) { k2 = idx % h2; q = idx / h2; } else { q = idx % h2; k2 = idx / h2; }
        Ys[k2 * h2 + q] = ld_fresh(Y + (size_t)k2 * yr + (size_t)q * yc);
    }
    __syncthreads();
    const int half = (h2 + 1) / 2;
    for (int t = threadIdx.x; t < half * half; t += blockDim.x) {
        const int p0 = 2 * (t / half), q0 = 2 * (t % half);
        T a00 = T(0), a01 = T(0), a10 = T(0), a11 = T(0);
        const bool p1 = p0 + 1 < h2, q1 = q0 + 1 < h2;
        for (int kk = 0; kk < h2; ++kk) {
            const T x0 = Xs[p0 * h2 + kk], x1 = p1 ? Xs[(p0 + 1) * h2 + kk] : T(0);
            const T y0 = Ys[kk * h2 + q0], y1 = q1 ? Ys[kk * h2 + q0 + 1] : T(0);
            a00 = fma(x0, y0, a00); a01 = fma(x0, y1, a01);
            a10 = fma(x1, y0, a10); a11 = fma(x1, y1, a11);
        }
        const T v[4] = {a00, a01, a10, a11};
        for (int e = 0; e < 4; ++e) {
            const int p = p0 + (e >> 1), q = q0 + (e & 1);
            if (p >= h2 || q >= h2) continue;
            T *o = out + (size_t)p * ldo + q;
            if (mode == 1) *o = ld_fresh(o) - v[e];
            else if (mode == 2) *o = -v[e];
            else *o = v[e];
        }
    }
    __syncthreads();
}

// Schur updates of the kept neighbours of each eliminated cell i at level l
// (s = 2^l), using only the N/2-wide coupling blocks:
//   right j = i+s:  A_j[L+,L-] -= B_j Ainv_i[R+,R-] C_i
//                   B_j' = -B_j Ainv_i[R+,L+] B_i
//   left  j = i-s:  A_j[R-,R+] -= C_j Ainv_i[L-,L+] B_i
//                   C_j' = -C_j Ainv_i[L-,R-] C_i   (0 if i has no right neighbour)
// Shared memory: 3 (N/2)^2 values (the product X and the staging buffer) when
// staged, else (N/2)^2 (X only; operands read from global memory).
template <typename T>
__device__ __forceinline__ void schur_body(T *__restrict__ A, T *__restrict__ Bc, T *__restrict__ Cc,
                                           const BcrItem &it, int N, int staged, unsigned char *smem_raw) {
    const int n2 = 2 * N, h2 = N / 2, hh = h2 * h2;
    T *X = reinterpret_cast<T *>(smem_raw);
    T *buf = staged ? X + hh : nullptr;
    const T *Ai = A + (size_t)it.cell * n2 * n2;  // transposed inverse: Ainv[r][c] = Ai[c*n2 + r]
    const int Lm = 0, Lp = h2, Rm = N, Rp = N + h2;
    const T *Bi = Bc + (size_t)it.s_cell * hh;
    const T *Ci = Cc + (size_t)it.s_cell * hh;
    // Ainv[r0 + p][c0 + k] = Ai[(c0 + k) * n2 + r0 + p]: row stride 1, col stride n2
    if (it.right >= 0) {
        const T *Bj = Bc + (size_t)it.s_right * hh;
        T *Aj = A + (size_t)it.right * n2 * n2;
        smem_mm(X, h2, 0, Bj, h2, 1, Ai + (size_t)Rm * n2 + Rp, 1, n2, h2, buf);   // X = B_j Ainv[R+,R-]
        smem_mm(Aj + (size_t)Lp * n2 + Lm, n2, 1, X, h2, 1, Ci, h2, 1, h2, buf);    // A_j[L+,L-] -= X C_i
        smem_mm(X, h2, 0, Bj, h2, 1, Ai + (size_t)Lp * n2 + Rp, 1, n2, h2, buf);   // X = B_j Ainv[R+,L+]
        smem_mm(Bc + (size_t)it.s_right_next * hh, h2, 2, X, h2, 1, Bi, h2, 1, h2, buf);  // B_j' = -X B_i
    }
    if (it.left >= 0) {
        const T *Cj = Cc + (size_t)it.s_left * hh;
        T *Aj = A + (size_t)it.left * n2 * n2;
        smem_mm(X, h2, 0, Cj, h2, 1, Ai + (size_t)Lp * n2 + Lm, 1, n2, h2, buf);   // X = C_j Ainv[L-,L+]
        smem_mm(Aj + (size_t)Rm * n2 + Rp, n2, 1, X, h2, 1, Bi, h2, 1, h2, buf);    // A_j[R-,R+] -= X B_i
        T *Cn = Cc + (size_t)it.s_left_next * hh;
        if (it.right >= 0) {
            smem_mm(X, h2, 0, Cj, h2, 1, Ai + (size_t)Rm * n2 + Lm, 1, n2, h2, buf);  // X = C_j Ainv[L-,R-]
            smem_mm(Cn, h2, 2, X, h2, 1, Ci, h2, 1, h2, buf);                         // C_j' = -X C_i
        } else {
            for (int idx = threadIdx.x; idx < hh; idx += blockDim.x) Cn[idx] = T(0);
        }
    }
}

template <typename T>
__global__ void k_bcr_schur(T *__restrict__ A, T *__restrict__ Bc, T *__restrict__ Cc,
                            const BcrItem *__restrict__ items, int N, int staged) {
    extern __shared__ unsigned char smem_raw[];
    schur_body(A, Bc, Cc, items[blockIdx.x], N, staged, smem_raw);
}

// ---------------------------------------------------------------------------
// Block cyclic reduction, solve F u = rhs for every rhs, in place.
// Forward (level l, eliminated i): y_i = Ainv_i r_i; r_{i+s}[L+] -= B_{i+s} y_i[R+];
// r_{i-s}[R-] -= C_{i-s} y_i[L-]. Roots: u = Ainv r.
// Backward (level l descending): u_i = y_i - Ainv_i[:,L+] B_i u_{i-s}[R+]
//                                          - Ainv_i[:,R-] C_i u_{i+s}[L-].
// One block per (item, rhs); every write touches a disjoint sub-vector.
// ---------------------------------------------------------------------------
// Row-sliced BCR solve units (push style). One BLOCK of NT threads handles one
// (item, rhs, row slice) unit; a level's units spread over all blocks, and at the
// upper levels (few items) an item's 2N rows are split into S in {1, 2, 4}
// slices so that several SMs share one matrix-vector product. With S <= 4 every
// slice boundary is a quadrant boundary (L-, L+, R-, R+ are N/2 rows each).
//   forward (item i at level l, s = 2^l, or a root):
//     y_i = A_i^{-1} r_i                                (rows of this slice) -> Y
//     the slice holding y_i[R+] pushes  r_{i+s}[L+] -= B_{i+s} y_i[R+]
//     the slice holding y_i[L-] pushes  r_{i-s}[R-] -= C_{i-s} y_i[L-]
//   backward (item i at level l, descending; u of the kept neighbours is final):
//     u_i = y_i - A_i^{-1}[:, L+] B_i u_{i-s}[R+] - A_i^{-1}[:, R-] C_i u_{i+s}[L-]
// r_i is complete when item i's level runs (its pushes came from lower levels);
// every pushed-to sub-vector has exactly one writer per level, so nothing races.
// rhs and Y are written by other blocks between grid-wide barriers and are read
// with L1-bypassing loads. The solution is left in Y.
template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    using type = float4;
    static constexpr int V = 4;
};
template <>
struct VecOf<double> {
    using type = double2;
    static constexpr int V = 2;
};

// Coupling blocks of one unit (the two N/2 x N/2 blocks it multiplies) are staged
// in shared memory by asynchronous copies issued when the unit starts, when both
// fit in 16 KB and a block is a whole number of 16-byte chunks.
__host__ __device__ constexpr int bcr_coupling_values(int N) { return 2 * (N / 2) * (N / 2); }
__host__ __device__ constexpr bool bcr_couplings_staged(int N, int esize) {
    return bcr_coupling_values(N) * esize <= 16384 && ((N / 2) * (N / 2) * esize) % 16 == 0;
}

// shared scratch (values of T) of one solve block handling RC right-hand sides:
// rs, ys (RC x 2N), pushed products (RC x N), partial sums (NT x V x RC), couplings
__host__ __device__ constexpr int bcr_unit_smem_values(int N, int NT, int V, int RC, int esize) {
    return RC * (2 * N) + RC * (2 * N) + RC * N + NT * V * RC + (bcr_couplings_staged(N, esize) ? bcr_coupling_values(N) : 0);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Start copying the coupling blocks m0, m1 (either may be NULL) into cbuf[0, hh) and
// cbuf[hh, 2 hh); returns the shared-memory copies (NULL where absent), or m0, m1
// themselves when cbuf is NULL (blocks read from global memory).
template <typename T>
__device__ __forceinline__ void stage_couplings(const T *&m0, const T *&m1, T *cbuf, int hh) {
    if (!cbuf) return;
    const int chunks = hh * (int)sizeof(T) / 16;
    for (int c = threadIdx.x; c < 2 * chunks; c += blockDim.x) {
        const int side = c >= chunks, cc = c - side * chunks;
        const T *src = side ? m1 : m0;
        if (src)
            cp_async16(reinterpret_cast<unsigned char *>(cbuf + side * hh) + 16 * cc,
                       reinterpret_cast<const unsigned char *>(src) + 16 * cc);
    }
    cp_async_commit();
    m0 = m0 ? cbuf : nullptr;
    m1 = m1 ? cbuf + hh : nullptr;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// For RC right-hand sides at once (coef[rc][k], row stride cstride):
// part[ks][rc][row] = sum over the k of slice ks of Mt[col(k)][row0 + row] * coef[rc][k],
// rows [row0, row0 + nr), col(k) = col_off0 + k for k < col_split else col_off1 + k - col_split.
// Each thread owns one (row group of V rows, k-slice) task and loads its A^{-1}
// vectors into registers in chunks of KC columns; the first chunk is requested
// BEFORE stage() runs (stage stages the coefficients and ends with a block
// barrier), so the factor reads overlap the wait for the right-hand side.
// Each A^{-1} vector is loaded once and used for all RC right-hand sides.
// Returns the number of k-slices. KC = 8: with 16 the unstaged solve kernels
// (2N = 256) spilled 236-748 bytes per thread at their 128-register cap, and the
// spill traffic serialised the factor stream (2.30 against 0.99 ms per solve
// launch, 0.29 against 0.67 of HBM, on the Batching recipe's N = 128 group).
constexpr int kMatvecChunk = 8;
template <typename T, int NT, int RC, typename Stage>
__device__ __forceinline__ int sliced_matvec(const T *__restrict__ Mt, int n2, int row0, int nr, int nk,
                                             int col_split, int col_off0, int col_off1, const T *coef, int cstride,
                                             T *part, Stage stage) {
    using VT = typename VecOf<T>::type;
    constexpr int V = VecOf<T>::V, KC = kMatvecChunk;
    const int RG = nr / V;
    int KS = NT / RG;
    if (KS > nk) KS = nk;
    if (KS < 1) KS = 1;
    const int kl = (nk + KS - 1) / KS;
    const int t = threadIdx.x;
    const bool act = t < RG * KS;  // RG * KS <= NT for nr <= V * NT
    const int rg = act ? t % RG : 0, ks = act ? t / RG : 0;
    const int k0 = ks * kl, k1 = act ? min(nk, k0 + kl) : k0;
    auto col_of = [&](int k) { return (k < col_split) ? col_off0 + k : col_off1 + (k - col_split); };
    VT a[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
        const int k = k0 + kk;
        if (k < k1) a[kk] = __ldg(reinterpret_cast<const VT *>(Mt + (size_t)col_of(k) * n2 + row0) + rg);
    }
    stage();
    T acc[RC][V];
#pragma unroll
    for (int rc = 0; rc < RC; ++rc)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[rc][v] = T(0);
    for (int c0 = k0; c0 < k1; c0 += KC) {
        if (c0 > k0) {
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                const int k = c0 + kk;
                if (k < k1) a[kk] = __ldg(reinterpret_cast<const VT *>(Mt + (size_t)col_of(k) * n2 + row0) + rg);
            }
        }
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            const int k = c0 + kk;
            if (k < k1) {
#pragma unroll
                for (int rc = 0; rc < RC; ++rc) {
                    const T cv = coef[rc * cstride + k];
                    if constexpr (V == 4) {
                        acc[rc][0] = fma(a[kk].x, cv, acc[rc][0]); acc[rc][1] = fma(a[kk].y, cv, acc[rc][1]);
                        acc[rc][2] = fma(a[kk].z, cv, acc[rc][2]); acc[rc][3] = fma(a[kk].w, cv, acc[rc][3]);
                    } else {
                        acc[rc][0] = fma(a[kk].x, cv, acc[rc][0]); acc[rc][1] = fma(a[kk].y, cv, acc[rc][1]);
                    }
                }
            }
        }
    }
    if (act) {
#pragma unroll
        for (int rc = 0; rc < RC; ++rc)
#pragma unroll
            for (int v = 0; v < V; ++v) part[(ks * RC + rc) * nr + rg * V + v] = acc[rc][v];
    }
    return KS;
}

// Up to two h2 x h2 coupling products for RC vectors at once, all NT threads:
// rows (side, p) of M_side (row-major), a group of G threads per row, each
// reading a contiguous k-range once for all RC vectors; partial sums meet by
// shuffles (M_side in global or shared memory). With nred = 0:
// out_side[rc * ostride + p] = sum_k M_side[p][k] v_side[rc * vstride + k]
// (shared memory). With nred > 0: out_side[rc * ostride + p] -= that sum for rc < nred, as a
// reduction without return in global memory.
template <typename T, int NT, int RC>
__device__ __forceinline__ void coupling_products(const T *__restrict__ M0, const T *v0, T *out0,
                                                  const T *__restrict__ M1, const T *v1, T *out1, int h2,
                                                  int vstride, size_t ostride, int nred = 0,
                                                  int tid = (int)threadIdx.x) {
    const int nrows = (M0 ? h2 : 0) + (M1 ? h2 : 0);
    if (nrows == 0) return;
    int G = 1;
    while (G < 32 && G * 2 * nrows <= NT && G * 2 <= h2) G *= 2;
    const int kl = (h2 + G - 1) / G;
    for (int t = tid; t < ((nrows * G + 31) & ~31); t += NT) {  // whole warps for the shuffles
        const int row = t / G, gq = t % G;
        const bool live = row < nrows;
        const bool second = live && (!M0 || row >= h2);
        const int p = second ? row - (M0 ? h2 : 0) : row;
        const T *M = second ? M1 : M0;
        const T *v = second ? v1 : v0;
        T acc[RC];
#pragma unroll
        for (int rc = 0; rc < RC; ++rc) acc[rc] = T(0);
        if (live) {
            const int k0 = gq * kl, k1 = min(h2, k0 + kl), len = k1 - k0;
            // each row starts its k-range at an offset of its own (p mod len): rows a
            // warp reads together then fall in different shared-memory banks
            int j = len > 0 ? p % len : 0;
#pragma unroll 4
            for (int c = 0; c < len; ++c) {
                const int k = k0 + j;
                j = (j + 1 == len) ? 0 : j + 1;
                const T m = M[(size_t)p * h2 + k];
#pragma unroll
                for (int rc = 0; rc < RC; ++rc) acc[rc] = fma(m, v[rc * vstride + k], acc[rc]);
            }
        }
#pragma unroll
        for (int rc = 0; rc < RC; ++rc) {
            const T s = group_sum(acc[rc], G);
            if (live && gq == 0) {
                T *o = (second ? out1 : out0) + rc * ostride + p;
                if (nred == 0) *o = s;
                else if (rc < nred) atomicAdd(o, -s);
            }
        }
    }
}

// Dataflow synchronisation of the BCR solve units (k_bcr_solve_flow): a unit waits
// until the counters it depends on reach their targets (thread 0 polls with acquire
// loads, at most `limit` times, then records *err = 1 and goes on), and after
// its writes (block barrier, then thread 0 fences) bumps the counters of the units
// that depend on it. NULL pointers are absent waits / signals.
// The limit is the context's: err[1] holds it (err[0] is the error flag), so a host
// can shorten it to make a wait run out on purpose (tests of the error path).
constexpr unsigned kFlowSpinLimit = 1u << 25;  // default: x >= 32 ns, about a second
__device__ __forceinline__ unsigned flow_spin_limit(const int *err) { return (unsigned)__ldg(err + 1); }
struct FlowSync {
    const int *wait0, *wait1;
    int want0, want1;
    int *sig0, *sig1, *sig2;
    int *err;
    unsigned limit;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void flow_wait(const FlowSync *fs) {
    if (!fs) return;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int *c = k ? fs->wait1 : fs->wait0;
            const int want = k ? fs->want1 : fs->want0;
            if (!c) continue;
            unsigned spins = 0;
            while (ld_acquire_gpu(c) < want) {  // busy first, then with short sleeps
                if (++spins > fs->limit) {
                    atomicExch(fs->err, 1);
                    break;
                }
                if (spins > 256) __nanosleep(32);
            }
        }
    }
    __syncthreads();
}

// The block barrier orders every thread's earlier writes before the signalling
// thread's fence, which then orders them before the counter bumps (the pattern of a
// cooperative grid barrier's arrival). The staged-slice solve signals from a thread
// outside warp 0 (thread 0 polls for the block's next unit meanwhile) with a
// release fence paired with the consumers' acquire loads; its units end without a
// second barrier (every read of the unit's scratch precedes the first one).
__device__ __forceinline__ void flow_signal(const FlowSync *fs) {
    if (!fs) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (fs->sig0) atomicAdd(fs->sig0, 1);
        if (fs->sig1) atomicAdd(fs->sig1, 1);
        if (fs->sig2) atomicAdd(fs->sig2, 1);
    }
}

__device__ __forceinline__ void flow_signal_release(const FlowSync *fs, int signaller) {
    if (!fs) return;
    __syncthreads();
    if ((int)threadIdx.x == signaller) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (fs->sig0) atomicAdd(fs->sig0, 1);
        if (fs->sig1) atomicAdd(fs->sig1, 1);
        if (fs->sig2) atomicAdd(fs->sig2, 1);
    }
}

// The factorization as a dataflow over the items of every level and the roots, in
// one cooperative launch of one 512-thread block per SM (register-tiled inversion,
// 2N in {32, 64, 128}). Items are taken block-stride in the order of the item array
// (levels ascending, roots last), and an item waits until its block has received
// every Schur update of the levels below its own: one from each neighbour at
// distance 2^l' for l' < its level, the count of the solve's pushes. It then inverts
// the block, applies its own Schur updates to its two kept neighbours (and their
// next-level couplings) and bumps their counters. A quadrant of a kept cell is
// updated by its neighbours at successive levels, each of which waited for the
// previous one, so plain read-modify-writes suffice; every read of data another
// block wrote bypasses L1. Waits are bounded (err[1] polls; *err = 1 on timeout).
template <typename T, int N2>
__global__ void __launch_bounds__(512, 1) k_bcr_factor_flow(T *__restrict__ A, const BcrItem *__restrict__ items,
                                                           int n_items, T *__restrict__ Bc, T *__restrict__ Cc,
                                                           unsigned long long *__restrict__ growth,
                                                           int *__restrict__ status, int *cnt, int *err,
                                                           int schur_staged) {
    extern __shared__ unsigned char smem_dyn[];
    const unsigned limit = flow_spin_limit(err);
    for (int ii = blockIdx.x; ii < n_items; ii += gridDim.x) {
        const BcrItem it = items[ii];
        FlowSync fs{};
        fs.err = err;
        fs.limit = limit;
        int want = 0;
        for (int lp = 0; lp < it.level; ++lp)
            want += (it.local >= (1 << lp)) + (it.local + (1 << lp) < it.K_inst);
        if (want) {
            fs.wait0 = cnt + it.cell;
            fs.want0 = want;
        }
        flow_wait(&fs);
        T *Ag = A + (size_t)it.cell * N2 * N2;
        if constexpr (sizeof(T) == 4) gj_panel_body<N2>(Ag, N2, Ag, N2, true, growth, status);
        else gj_reg_body<T, N2>(Ag, N2, Ag, N2, true, growth, status);
        if (it.left >= 0 || it.right >= 0) {
            __syncthreads();  // the inverse this block just wrote, before the updates read it
            schur_body(A, Bc, Cc, it, N2 / 2, schur_staged, smem_dyn);
            if (it.right >= 0) fs.sig0 = cnt + it.right;
            if (it.left >= 0) fs.sig1 = cnt + it.left;
            flow_signal(&fs);
        }
        __syncthreads();  // shared memory of the inversion reused by the block's next item
    }
}

// Units cover RC consecutive right-hand sides r0 .. r0 + nrc - 1 (nrc <= RC).
template <typename T, int NT, int RC>
__device__ __forceinline__ void bcr_fwd_unit(const T *__restrict__ A, const T *__restrict__ Bc,
                                             const T *__restrict__ Cc, const BcrItem &it, int r0, int nrc, int sl,
                                             int S, T *rhs, T *Y, int N, int sumK, T *sm,
                                             const FlowSync *fs = nullptr) {
    const int n2 = 2 * N, h2 = N / 2, hh = h2 * h2;
    T *rs = sm, *ys = sm + RC * n2, *part = ys + RC * n2 + RC * N;
    T *cbuf = bcr_couplings_staged(N, (int)sizeof(T)) ? part + NT * VecOf<T>::V * RC : nullptr;
    const size_t rstride = (size_t)sumK * n2;  // between right-hand sides
    const int nr = n2 / S, row0 = sl * nr;
    const T *Ai = A + (size_t)it.cell * n2 * n2;
    const bool push_right = it.right >= 0 && row0 + nr == n2;  // this slice holds R+
    const bool push_left = it.left >= 0 && row0 == 0;          // this slice holds L-
    const T *mB = push_right ? Bc + (size_t)it.s_right * hh : nullptr;
    const T *mC = push_left ? Cc + (size_t)it.s_left * hh : nullptr;
    stage_couplings(mB, mC, cbuf, hh);  // in flight during the matrix-vector product
    const int KS = sliced_matvec<T, NT, RC>(Ai, n2, row0, nr, n2, n2, 0, 0, rs, n2, part, [&] {
        flow_wait(fs);  // r_i complete (every push into it has landed)
        for (int i = threadIdx.x; i < RC * n2; i += NT) {
            const int rc = i / n2, k = i - rc * n2;
            rs[i] = rc < nrc ? __ldcg(rhs + (size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + k) : T(0);
        }
        __syncthreads();
    });
    __syncthreads();
    for (int idx = threadIdx.x; idx < RC * nr; idx += NT) {
        const int rc = idx / nr, row = idx - rc * nr;
        T y = T(0);
        for (int s = 0; s < KS; ++s) y += part[(s * RC + rc) * nr + row];
        ys[rc * n2 + row0 + row] = y;
        if (rc < nrc) Y[(size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + row0 + row] = y;
    }
    if (cbuf) cp_async_wait_all();
    __syncthreads();
    // pushes as reductions without return (one writer per sub-vector and level, so
    // old - product is formed exactly as a read-modify-write would)
    coupling_products<T, NT, RC>(mB, ys + N + h2,
                                 push_right ? rhs + (size_t)r0 * rstride + (size_t)it.right * n2 + h2 : nullptr,
                                 mC, ys, push_left ? rhs + (size_t)r0 * rstride + (size_t)it.left * n2 + N : nullptr,
                                 h2, n2, rstride, nrc);
    flow_signal(fs);
    __syncthreads();  // scratch reuse by the block's next unit
}

template <typename T, int NT, int RC>
__device__ __forceinline__ void bcr_bwd_unit(const T *__restrict__ A, const T *__restrict__ Bc,
                                             const T *__restrict__ Cc, const BcrItem &it, int r0, int nrc, int sl,
                                             int S, T *Y, int N, int sumK, T *sm, const FlowSync *fs = nullptr) {
    const int n2 = 2 * N, h2 = N / 2, hh = h2 * h2;
    T *gv = sm, *g = sm + RC * N, *part = sm + RC * (5 * N);  // gv[rc] = [u_left[R+], u_right[L-]]
    T *cbuf = bcr_couplings_staged(N, (int)sizeof(T)) ? part + NT * VecOf<T>::V * RC : nullptr;
    const size_t rstride = (size_t)sumK * n2;
    const int nr = n2 / S, row0 = sl * nr;
    const T *Ai = A + (size_t)it.cell * n2 * n2;
    const T *mB = Bc + (size_t)it.s_cell * hh, *mC = it.right >= 0 ? Cc + (size_t)it.s_cell * hh : nullptr;
    stage_couplings(mB, mC, cbuf, hh);
    const int KS = sliced_matvec<T, NT, RC>(Ai, n2, row0, nr, N, h2, h2, N, g, N, part, [&] {
        flow_wait(fs);  // u of both kept neighbours final
        for (int idx = threadIdx.x; idx < RC * N; idx += NT) {
            const int rc = idx / N, k = idx - rc * N;
            T v = T(0);
            if (rc < nrc) {
                const T *base = Y + (size_t)(r0 + rc) * rstride;
                if (k < h2) v = __ldcg(base + (size_t)it.left * n2 + N + h2 + k);
                else if (it.right >= 0) v = __ldcg(base + (size_t)it.right * n2 + (k - h2));
            }
            gv[idx] = v;
        }
        if (cbuf) cp_async_wait_all();
        __syncthreads();
        coupling_products<T, NT, RC>(mB, gv, g, mC, gv + h2, g + h2, h2, N, N);
        if (it.right < 0)
            for (int idx = threadIdx.x; idx < RC * h2; idx += NT) g[(idx / h2) * N + h2 + idx % h2] = T(0);
        __syncthreads();
    });
    __syncthreads();
    for (int idx = threadIdx.x; idx < nrc * nr; idx += NT) {
        const int rc = idx / nr, row = idx - rc * nr;
        T s = T(0);
        for (int q = 0; q < KS; ++q) s += part[(q * RC + rc) * nr + row];
        atomicAdd(Y + (size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + row0 + row, -s);
    }
    flow_signal(fs);
    __syncthreads();
}

// Item ranges of every reduction level in one concatenated item array:
// level l owns items [off[l], off[l+1]); roots follow at [off[n_levels], off[n_levels] + n_roots).
// slices[l] = row slices per item at level l (index n_levels: the roots).
constexpr int kMaxLevels = 32;
// Coarse step (staged-slice solve of a single instance and right-hand side only):
// with coarse_level = c >= 0 the levels c .. n_levels - 1 and the root are replaced
// by u_c = G r_c, G the inverse of the block-tridiagonal system that the reduction
// leaves on the coarse cells (local index a multiple of 2^c, coarse_m of them,
// coarse_K cells in the instance), computed once per factorization. G rows are
// taken coarse_rpu at a time by coarse_units units. coarse_level = -1: no coarse step.
struct LevelTable {
    int32_t off[kMaxLevels + 2];
    int32_t slices[kMaxLevels + 2];
    int32_t n_levels, n_roots;
    int32_t coarse_level, coarse_m, coarse_K, coarse_rpu, coarse_units;
    int32_t n_stages;  // staged-slice solve: copy stages per block (1 .. kMaxSolveStages)
};

// The BCR solve as a dataflow over all units in one cooperative launch, without
// grid-wide barriers. Units are numbered phase by phase (forward levels, roots,
// backward levels) and taken block-stride in that order, so every unit depends only
// on units numbered before it and, all blocks being co-resident, every wait ends.
// Counters per (right-hand-side chunk, cell), zero at launch:
//   cnt[ch][i]   pushes landed in r_i; the forward unit of item i at level l (local
//                index a, instance size K) waits for sum_{l' < l} ([a >= 2^l'] + [a + 2^l' < K])
//   done[ch][i]  slices of cell i whose u is final (its root solve or backward update);
//                the backward unit of item i waits for all slices of both kept neighbours
// A unit requests its A^{-1} vectors before it waits, so the factor reads overlap the
// wait. The levels thus overlap: a unit starts as soon as its own inputs are final.
__device__ __forceinline__ int bcr_cell_level(int local, int n_levels) {
    return local == 0 ? n_levels : __ffs(local) - 1;
}

template <typename T, int NT, int RC>
__global__ void __launch_bounds__(NT, 2) k_bcr_solve_flow(const T *__restrict__ A, const T *__restrict__ Bc,
                                                       const T *__restrict__ Cc, const BcrItem *__restrict__ items,
                                                       LevelTable lv, T *rhs, T *Y, int N, int sumK, int R, int *cnt,
                                                       int *done, int *err,
                                                       const T *__restrict__ G /* coarse step: staged only */,
                                                       int *zero_next, long long nzero) {
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < nzero; i += (long long)gridDim.x * NT)
        zero_next[i] = 0;
    tc::grid_dependency_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const unsigned limit = flow_spin_limit(err);
    const int nchunk = (R + RC - 1) / RC, nl = lv.n_levels, P = 2 * nl;
    auto phase_level = [&](int ph) { return ph <= nl ? ph : 2 * nl - ph; };
    auto units = [&](int ph) {
        const int l = phase_level(ph);
        const int nitems = (l < nl) ? lv.off[l + 1] - lv.off[l] : lv.n_roots;
        return nitems * nchunk * lv.slices[l];
    };
    int ph = 0, start = 0;  // phase of the current unit and its first global index
    for (int gidx = blockIdx.x;; gidx += gridDim.x) {
        while (ph <= P && gidx >= start + units(ph)) {
            start += units(ph);
            ++ph;
        }
        if (ph > P) break;
        const int l = phase_level(ph), S = lv.slices[l], w = gidx - start;
        const int sl = w % S, ch = (w / S) % nchunk, item = w / (S * nchunk);
        const int r0 = ch * RC, nrc = min(RC, R - r0);
        const BcrItem it = items[lv.off[l] + item];
        int *cnt_c = cnt + (size_t)ch * sumK, *done_c = done + (size_t)ch * sumK;
        const int n2 = 2 * N, nr = n2 / S, row0 = sl * nr;
        FlowSync fs{};
        fs.err = err;
        fs.limit = limit;
        if (ph <= nl) {
            int want = 0;
            for (int lp = 0; lp < it.level; ++lp)
                want += (it.local >= (1 << lp)) + (it.local + (1 << lp) < it.K_inst);
            if (want) {
                fs.wait0 = cnt_c + it.cell;
                fs.want0 = want;
            }
            if (it.right >= 0 && row0 + nr == n2) fs.sig0 = cnt_c + it.right;
            if (it.left >= 0 && row0 == 0) fs.sig1 = cnt_c + it.left;
            if (it.left < 0) fs.sig2 = done_c + it.cell;  // a root: its solution is final
            bcr_fwd_unit<T, NT, RC>(A, Bc, Cc, it, r0, nrc, sl, S, rhs, Y, N, sumK, sm, &fs);
        } else {
            const int step = 1 << it.level;
            fs.wait0 = done_c + it.left;
            fs.want0 = lv.slices[bcr_cell_level(it.local - step, nl)];
            if (it.right >= 0) {
                fs.wait1 = done_c + it.right;
                fs.want1 = lv.slices[bcr_cell_level(it.local + step, nl)];
            }
            fs.sig0 = done_c + it.cell;
            bcr_bwd_unit<T, NT, RC>(A, Bc, Cc, it, r0, nrc, sl, S, Y, N, sumK, sm, &fs);
        }
    }
}

// ---------------------------------------------------------------------------
// Shared-memory staged variant of the dataflow BCR solve (used when a cell's whole
// A^{-1} fits in kSolveStageBytes): the columns a unit multiplies (one contiguous
// block of the transposed inverse) and its two coupling blocks are copied into
// shared memory by bulk asynchronous copies (the TMA engine: three instructions of
// one thread instead of thousands of 16-byte copies, which backed up the load/store
// path while the wide levels stream), and the copy for the block's NEXT unit is
// issued as soon as the current unit's matrix-vector product has read its columns,
// so a block's factor stream overlaps the unit's reduction, pushes, fence and
// counter bump and the next unit's wait for its inputs. The coupling blocks are
// double-buffered (the current unit multiplies by them after the next copy starts).
// ---------------------------------------------------------------------------
constexpr int kSolveStageBytes = 64 * 1024;

__host__ __device__ constexpr bool bcr_slice_staged(int N, int esize) {
    return (size_t)(2 * N) * (2 * N) * esize <= (size_t)kSolveStageBytes && (2 * N * esize) % 16 == 0;
}

// Shared memory of a staged-slice solve block: the unit scratch, then n_stages copy
// stages, each one unit's A^{-1} columns ((2N)^2 values) followed by its coupling
// area (2 (N/2)^2 values, when the couplings are staged; a coarse unit's r_c there),
// every area starting on a 16-byte boundary.
constexpr int kMaxSolveStages = 4;
// values of T filling whole 16-byte chunks, at least v
template <typename T>
__host__ __device__ constexpr int bcr_round16(int v) {
    return (v * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
}
template <typename T>
__host__ __device__ constexpr int bcr_stage_base_values(int N, int NT, int RC) {
    return bcr_round16<T>(bcr_unit_smem_values(N, NT, VecOf<T>::V, RC, (int)sizeof(T)) -
                          (bcr_couplings_staged(N, (int)sizeof(T)) ? bcr_coupling_values(N) : 0));
}
// one stage: the A^{-1} columns, the coupling area, and the right-hand sides of a
// unit whose inputs are known at issue time (RC x 2N values)
template <typename T>
__host__ __device__ constexpr int bcr_stage_rhs_offset(int N) {
    return bcr_round16<T>((2 * N) * (2 * N) + (bcr_couplings_staged(N, (int)sizeof(T)) ? bcr_coupling_values(N) : 0));
}
template <typename T>
__host__ __device__ constexpr int bcr_stage_values(int N, int RC) {
    return bcr_stage_rhs_offset<T>(N) + bcr_round16<T>(RC * 2 * N);
}

// The coupling blocks a unit multiplies (global memory; NULL where absent): forward
// units push through B (right neighbour, from the slice holding R+) and C (left
// neighbour, from the slice holding L-); backward units multiply the kept
// neighbours' solutions by the cell's own B and C.
template <typename T>
__device__ __forceinline__ void unit_coupling_sources(const BcrItem &it, int sl, int S, bool bwd, int N,
                                                      const T *Bc, const T *Cc, const T *&m0, const T *&m1) {
    const int n2 = 2 * N, hh = (N / 2) * (N / 2), nr = n2 / S, row0 = sl * nr;
    if (!bwd) {
        m0 = (it.right >= 0 && row0 + nr == n2) ? Bc + (size_t)it.s_right * hh : nullptr;
        m1 = (it.left >= 0 && row0 == 0) ? Cc + (size_t)it.s_left * hh : nullptr;
    } else {
        m0 = Bc + (size_t)it.s_cell * hh;
        m1 = it.right >= 0 ? Cc + (size_t)it.s_cell * hh : nullptr;
    }
}

// Copy the columns of the transposed inverse that unit (it, bwd) multiplies into
// As[k][row] (all 2N rows, k over the unit's columns in matvec order; forward: all
// 2N columns, backward: columns N/2 .. 3N/2 - 1, one contiguous block either way)
// and, with cb, its coupling blocks into cb[0, hh) and cb[hh, 2 hh), by bulk
// asynchronous copies (the TMA engine) that complete one phase of *bar. A unit with
// a row slice reads its rows of the block. Issued by one warp (the block's last:
// thread 0, which fences the unit's signal, is not held up by the copies). Every
// address and size is a multiple of 16 bytes (rows of 2N values of whole 16-byte
// vectors; N/2 x N/2 coupling blocks staged only when whole 16-byte chunks).
template <typename T>
__device__ __forceinline__ void stage_unit_bulk(const T *__restrict__ A, const T *__restrict__ Bc,
                                                const T *__restrict__ Cc, const BcrItem &it, int sl, int S, bool bwd,
                                                int N, T *As, T *cb, uint64_t *bar) {
    const int lane = threadIdx.x & 31;
    const int n2 = 2 * N, h2 = N / 2, nk = bwd ? N : n2;
    const T *m0 = nullptr, *m1 = nullptr;
    if (cb) unit_coupling_sources(it, sl, S, bwd, N, Bc, Cc, m0, m1);
    const uint32_t hb = (uint32_t)(h2 * h2 * sizeof(T)), sb = (uint32_t)((size_t)nk * n2 * sizeof(T));
    tc::fence_async_smem();  // the buffers' earlier generic reads before the copies' writes
    if (lane == 0) {
        tc::mbar_arrive_expect_tx(bar, sb + (m0 ? hb : 0u) + (m1 ? hb : 0u));
        if (m0) tc::bulk_copy_g2s(cb, m0, hb, bar);
        if (m1) tc::bulk_copy_g2s(cb + h2 * h2, m1, hb, bar);
        tc::bulk_copy_g2s(As, A + (size_t)it.cell * n2 * n2 + (bwd ? (size_t)h2 * n2 : 0), sb, bar);
    }
}

// part[ks][rc][row] for this thread's (row group, k-slice) task: rows [0, nr) of the staged
// A^{-1} columns As[k * lda + row] (shared memory).
template <typename T, int NT, int RC>
__device__ __forceinline__ int smem_matvec(const T *As, int lda, int nr, int nk, const T *coef, int cstride, T *part,
                                           int tid = (int)threadIdx.x) {
    using VT = typename VecOf<T>::type;
    constexpr int V = VecOf<T>::V;
    const int RG = nr / V;
    int KS = NT / RG;
    if (KS > nk) KS = nk;
    if (KS < 1) KS = 1;
    const int kl = (nk + KS - 1) / KS;
    const int t = tid;
    if (t < RG * KS) {
        const int rg = t % RG, ks = t / RG;
        const int k0 = ks * kl, k1 = min(nk, k0 + kl);
        T acc[RC][V];
#pragma unroll
        for (int rc = 0; rc < RC; ++rc)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[rc][v] = T(0);
#pragma unroll 8
        for (int k = k0; k < k1; ++k) {
            const VT a = *reinterpret_cast<const VT *>(As + (size_t)k * lda + rg * V);
#pragma unroll
            for (int rc = 0; rc < RC; ++rc) {
                const T cv = coef[rc * cstride + k];
                if constexpr (V == 4) {
                    acc[rc][0] = fma(a.x, cv, acc[rc][0]); acc[rc][1] = fma(a.y, cv, acc[rc][1]);
                    acc[rc][2] = fma(a.z, cv, acc[rc][2]); acc[rc][3] = fma(a.w, cv, acc[rc][3]);
                } else {
                    acc[rc][0] = fma(a.x, cv, acc[rc][0]); acc[rc][1] = fma(a.y, cv, acc[rc][1]);
                }
            }
        }
#pragma unroll
        for (int rc = 0; rc < RC; ++rc)
#pragma unroll
            for (int v = 0; v < V; ++v) part[(ks * RC + rc) * nr + rg * V + v] = acc[rc][v];
    }
    return KS;
}

// ---------------------------------------------------------------------------
// Warp roles of the staged solve: two compute groups of NTG threads (4 warps each)
// and two service warps. Group g computes the block's units k = g, g + 2, ... and
// synchronises on its own named barrier (1 + g); when it has finished a unit it only
// ARRIVES on the unit's handoff barrier (id 3 + (k mod n_stages) + n_stages g, NTG + 32
// threads) and goes on, while service warp g waits there, fences and bumps the
// counters of the units that depend on this one (the release fence's latency is off
// the compute path), then refills the unit's stage with the unit n_stages ahead. A stage's
// next fill is issued only after its unit has been handed off, and a group waits for a
// fill only once a service warp has published that it was issued (s_fills): so every
// earlier phase of the stage's mbarrier has completed (its parity then names the right
// phase), and a handoff barrier is arrived at again only after its previous round has
// completed. Two groups keep two units' latencies (input counters, right-hand-side
// loads) in flight on the SM, two service warps two fences.
constexpr int kSolveGroups = 2;
__device__ __forceinline__ void gbar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ bool gbar_or(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void handoff_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The thread indices and barrier of one compute group.
struct Group {
    int gt;   // thread index within the group
    int bar;  // named barrier id of the group
};

// A unit's input wait on a compute group: its thread 0 polls (bounded), then the group barrier.
template <int NTG>
__device__ __forceinline__ void flow_wait_g(const FlowSync *fs, const Group &gr) {
    if (gr.gt == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int *c = k ? fs->wait1 : fs->wait0;
            const int want = k ? fs->want1 : fs->want0;
            if (!c) continue;
            unsigned spins = 0;
            while (ld_acquire_gpu(c) < want) {
                if (++spins > fs->limit) {
                    atomicExch(fs->err, 1);
                    break;
                }
                if (spins > 256) __nanosleep(32);
            }
        }
    }
    gbar_sync(gr.bar, NTG);
}

// Forward / backward unit on a compute group, its A^{-1} slice in As and its coupling
// blocks (mB, mC: shared-memory copies, or global memory when not staged; NULL where
// absent) in flight; wait_copies() returns (true) once they have landed. The unit's
// results are written when it returns; its signal is the service warp's.
template <typename T, int NTG, int RC, typename WaitCopies>
__device__ __forceinline__ bool ring_fwd_unit(const T *mB, const T *mC, const BcrItem &it, int r0, int nrc, int sl,
                                              int S, T *rhs, T *Y, int N, int sumK, T *sm, const T *As,
                                              const T *rs_staged, const FlowSync *fs, const Group &gr,
                                              WaitCopies wait_copies) {
    const int n2 = 2 * N, h2 = N / 2, gt = gr.gt;
    T *ys = sm + RC * n2, *part = ys + RC * n2 + RC * N;
    const T *rs = rs_staged ? rs_staged : sm;  // right-hand sides staged with the unit's copies, or loaded here
    const size_t rstride = (size_t)sumK * n2;
    const int nr = n2 / S, row0 = sl * nr;
    if (!rs_staged) {
        flow_wait_g<NTG>(fs, gr);
        for (int i = gt; i < RC * n2; i += NTG) {
            const int rc = i / n2, k = i - rc * n2;
            sm[i] = rc < nrc ? __ldcg(rhs + (size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + k) : T(0);
        }
    }
    if (!wait_copies()) return false;  // a group barrier: rs complete too
    const int KS = smem_matvec<T, NTG, RC>(As + row0, n2, nr, n2, rs, n2, part, gt);
    gbar_sync(gr.bar, NTG);
    for (int idx = gt; idx < RC * nr; idx += NTG) {
        const int rc = idx / nr, row = idx - rc * nr;
        T y = T(0);
        for (int q = 0; q < KS; ++q) y += part[(q * RC + rc) * nr + row];
        ys[rc * n2 + row0 + row] = y;
        if (rc < nrc) Y[(size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + row0 + row] = y;
    }
    gbar_sync(gr.bar, NTG);
    coupling_products<T, NTG, RC>(mB, ys + N + h2,
                                  mB ? rhs + (size_t)r0 * rstride + (size_t)it.right * n2 + h2 : nullptr, mC, ys,
                                  mC ? rhs + (size_t)r0 * rstride + (size_t)it.left * n2 + N : nullptr, h2, n2,
                                  rstride, nrc, gt);
    return true;
}

template <typename T, int NTG, int RC, typename WaitCopies>
__device__ __forceinline__ bool ring_bwd_unit(const T *mB, const T *mC, const BcrItem &it, int r0, int nrc, int sl,
                                              int S, T *Y, int N, int sumK, T *sm, const T *As, const FlowSync *fs,
                                              const Group &gr, WaitCopies wait_copies) {
    const int n2 = 2 * N, h2 = N / 2, gt = gr.gt;
    T *gv = sm, *g = sm + RC * N, *part = sm + RC * (5 * N);
    const size_t rstride = (size_t)sumK * n2;
    const int nr = n2 / S, row0 = sl * nr;
    flow_wait_g<NTG>(fs, gr);
    for (int idx = gt; idx < RC * N; idx += NTG) {
        const int rc = idx / N, k = idx - rc * N;
        T v = T(0);
        if (rc < nrc) {
            const T *base = Y + (size_t)(r0 + rc) * rstride;
            if (k < h2) v = __ldcg(base + (size_t)it.left * n2 + N + h2 + k);
            else if (it.right >= 0) v = __ldcg(base + (size_t)it.right * n2 + (k - h2));
        }
        gv[idx] = v;
    }
    if (!wait_copies()) return false;
    coupling_products<T, NTG, RC>(mB, gv, g, mC, gv + h2, g + h2, h2, N, N, 0, gt);
    if (it.right < 0)
        for (int idx = gt; idx < RC * h2; idx += NTG) g[(idx / h2) * N + h2 + idx % h2] = T(0);
    gbar_sync(gr.bar, NTG);
    const int KS = smem_matvec<T, NTG, RC>(As + row0, n2, nr, N, g, N, part, gt);
    gbar_sync(gr.bar, NTG);
    for (int idx = gt; idx < nrc * nr; idx += NTG) {
        const int rc = idx / nr, row = idx - rc * nr;
        T sacc = T(0);
        for (int q = 0; q < KS; ++q) sacc += part[(q * RC + rc) * nr + row];
        atomicAdd(Y + (size_t)(r0 + rc) * rstride + (size_t)it.cell * n2 + row0 + row, -sacc);
    }
    return true;
}

// The coarse unit u on a compute group: rows [u rpu, (u + 1) rpu) of u_c = G r_c (G
// rows staged in As by the unit's bulk copy; r_c, the right-hand sides of the m coarse
// cells in coarse order, gathered into rc) once every coarse cell has received the
// pushes of the levels below c; the rows are written to Y.
template <typename T, int NTG, typename WaitCopies>
__device__ __forceinline__ bool ring_coarse_unit(int u, const LevelTable &lv, const T *rhs, T *Y, int N, T *rc,
                                                 const T *As, const int *cnt, int *err, unsigned limit,
                                                 const Group &gr, WaitCopies wait_copies) {
    const int n2 = 2 * N, cl = lv.coarse_level, m = lv.coarse_m, n = m * n2, rpu = lv.coarse_rpu, gt = gr.gt;
    for (int j = gt; j < m; j += NTG) {  // one poller per coarse cell
        const int a = j << cl;
        int want = 0;
        for (int lp = 0; lp < cl; ++lp) want += (a >= (1 << lp)) + (a + (1 << lp) < lv.coarse_K);
        unsigned spins = 0;
        while (want && ld_acquire_gpu(cnt + a) < want) {
            if (++spins > limit) {
                atomicExch(err, 1);
                break;
            }
            if (spins > 256) __nanosleep(32);
        }
    }
    gbar_sync(gr.bar, NTG);
    for (int idx = gt; idx < n; idx += NTG) {
        const int j = idx / n2;
        rc[idx] = __ldcg(rhs + (size_t)(j << cl) * n2 + (idx - j * n2));
    }
    if (!wait_copies()) return false;
    const int lane = gt & 31;
    for (int rr = gt >> 5; rr < rpu; rr += NTG / 32) {
        const T *g = As + (size_t)rr * n;
        T acc = T(0);
        for (int col = lane; col < n; col += 32) acc = fma(g[col], rc[col], acc);
        acc = group_sum(acc, 32);
        if (lane == 0) {
            const int row = u * rpu + rr, j = row / n2;
            Y[(size_t)(j << cl) * n2 + (row - j * n2)] = acc;
        }
    }
    return true;
}

// The dataflow BCR solve with staged slices (same unit order, counters and waits as
// k_bcr_solve_flow; with a coarse step, the levels from coarse_level up and the
// root are one phase of coarse units between the forward and backward levels below
// it). Shared memory: one unit scratch per compute group, then lv.n_stages copy
// stages. The factor columns, couplings and rows of G a unit reads do not change
// during the solve, so a block requests them lv.n_stages units ahead of the unit it
// computes (a ring: unit k of the block uses stage k mod n_stages, refilled with unit
// k + n_stages once unit k has been handed off); the copies thus stream while the
// compute groups wait for their units' inputs, and the dataflow waits only order the
// right-hand sides. The right-hand sides of level-0 forward units (the kernel's
// input, no dependencies) travel with their stage's copies, except for the first
// n_stages units, requested before the previous kernel has finished.
// NT = kSolveGroups compute groups of NTG threads + kSolveGroups service warps; service
// warp g hands off, signals and refills the units of group g.
template <typename T, int NT, int RC>
__global__ void __launch_bounds__(NT, 1) k_bcr_solve_flow_s(const T *__restrict__ A, const T *__restrict__ Bc,
                                                            const T *__restrict__ Cc,
                                                            const BcrItem *__restrict__ items, LevelTable lv, T *rhs,
                                                            T *Y, int N, int sumK, int R, int *cnt, int *done,
                                                            int *err, const T *__restrict__ G, int *zero_next,
                                                            long long nzero) {
    constexpr int NTG = (NT - 32 * kSolveGroups) / kSolveGroups;
    static_assert(NTG >= 64 && NTG % 32 == 0 && NT == kSolveGroups * (NTG + 32), "compute groups and service warps");
    // the next solve's counters (the other half of the double-buffered pair) start at zero
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < nzero; i += (long long)gridDim.x * NT)
        zero_next[i] = 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[kMaxSolveStages];  // per stage: one phase per fill
    __shared__ int s_fills[kMaxSolveStages];                   // per stage: fills issued so far
    __shared__ int s_stop;                                     // a compute group stopped (copy timeout)
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int hh = (N / 2) * (N / 2), n2 = 2 * N;
    const bool cpl_staged = bcr_couplings_staged(N, (int)sizeof(T));
    const int ns = lv.n_stages, base = bcr_stage_base_values<T>(N, NTG, RC);
    const size_t rstride = (size_t)sumK * n2;
    auto stage_slice = [&](int st) { return sm + kSolveGroups * base + st * bcr_stage_values<T>(N, RC); };
    auto stage_cpl = [&](int st) { return cpl_staged ? stage_slice(st) + n2 * n2 : (T *)nullptr; };
    auto stage_rhs = [&](int st) { return stage_slice(st) + bcr_stage_rhs_offset<T>(N); };
    if (threadIdx.x == 0) {
        for (int st = 0; st < ns; ++st) {
            tc::mbar_init(&s_bar[st], 1);
            s_fills[st] = 0;
        }
        s_stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nchunk = (R + RC - 1) / RC, nl = lv.n_levels, cl = lv.coarse_level;
    const int P = cl >= 0 ? 2 * cl : 2 * nl;
    const unsigned limit = flow_spin_limit(err);
    // level of a phase (-1: the coarse phase) and whether it is a backward phase
    auto phase_level = [&](int ph) {
        if (cl >= 0) return ph < cl ? ph : (ph == cl ? -1 : 2 * cl - ph);
        return ph <= nl ? ph : 2 * nl - ph;
    };
    auto phase_bwd = [&](int ph) { return cl >= 0 ? ph > cl : ph > nl; };
    auto units = [&](int ph) {
        const int l = phase_level(ph);
        if (l < 0) return lv.coarse_units;
        const int nitems = (l < nl) ? lv.off[l + 1] - lv.off[l] : lv.n_roots;
        return nitems * nchunk * lv.slices[l];
    };
    // units that complete a cell of the given level (its row slices, or the coarse units over its rows)
    auto done_want = [&](int level) { return (cl >= 0 && level >= cl) ? 2 * N / lv.coarse_rpu : lv.slices[level]; };
    struct Pos {
        int ph, start, l, S, sl, ch, item;
        bool valid;
    };
    auto locate = [&](Pos &q, int gidx) {
        while (q.ph <= P && gidx >= q.start + units(q.ph)) {
            q.start += units(q.ph);
            ++q.ph;
        }
        q.valid = q.ph <= P;
        if (!q.valid) return;
        q.l = phase_level(q.ph);
        const int w = gidx - q.start;
        if (q.l < 0) {  // coarse unit w
            q.S = 1;
            q.sl = 0;
            q.ch = 0;
            q.item = w;
            return;
        }
        q.S = lv.slices[q.l];
        q.sl = w % q.S;
        q.ch = (w / q.S) % nchunk;
        q.item = w / (q.S * nchunk);
    };
    // unit k of the block (at q) gets its right-hand sides with its copies: a level-0
    // forward unit requested after the previous kernel has finished, all RC rhs present
    auto rhs_staged = [&](const Pos &q, int k) {
        return k >= ns && q.l == 0 && !phase_bwd(q.ph) && (q.ch + 1) * RC <= R;
    };
    constexpr int kHandoff = NTG + 32;  // threads of a handoff barrier: one group and its service warp
    if (threadIdx.x >= kSolveGroups * NTG) {
        // ---- service warps: copies into the ring, then per unit: handoff, refill, signal
        const int sw = (threadIdx.x - kSolveGroups * NTG) >> 5, lane = threadIdx.x & 31;
        // copies of unit k into its stage (q located at k)
        auto issue = [&](const Pos &q, int k) {
            const int st = k % ns;
            if (q.l < 0) {
                const int n = lv.coarse_m * n2, rpu = lv.coarse_rpu;
                tc::fence_async_smem();
                if (lane == 0) {
                    const uint32_t bytes = (uint32_t)((size_t)rpu * n * sizeof(T));
                    tc::mbar_arrive_expect_tx(&s_bar[st], bytes);
                    tc::bulk_copy_g2s(stage_slice(st), G + (size_t)q.item * rpu * n, bytes, &s_bar[st]);
                }
            } else {
                const BcrItem itq = items[lv.off[q.l] + q.item];
                if (rhs_staged(q, k) && lane == 0) {
                    // the rhs copies join the phase before stage_unit_bulk's arrival
                    const uint32_t rb = (uint32_t)(n2 * sizeof(T));
                    tc::mbar_expect_tx(&s_bar[st], RC * rb);
                    for (int rc = 0; rc < RC; ++rc)
                        tc::bulk_copy_g2s(stage_rhs(st) + rc * n2,
                                          rhs + (size_t)(q.ch * RC + rc) * rstride + (size_t)itq.cell * n2, rb,
                                          &s_bar[st]);
                }
                stage_unit_bulk<T>(A, Bc, Cc, itq, q.sl, q.S, phase_bwd(q.ph), N, stage_slice(st), stage_cpl(st),
                                   &s_bar[st]);
            }
            __syncwarp();
            if (lane == 0) *(volatile int *)&s_fills[st] = k / ns + 1;
        };
        if (sw == 0) {  // factors, couplings and G are not written by the previous kernel
            Pos q{0, 0, 0, 0, 0, 0, 0, false};
            for (int k = 0; k < ns; ++k) {
                locate(q, blockIdx.x + k * (int)gridDim.x);
                if (q.valid) issue(q, k);
            }
        }
        tc::grid_dependency_wait();  // later copies may carry the previous kernel's right-hand sides
        Pos cur{0, 0, 0, 0, 0, 0, 0, false}, nxt{0, 0, 0, 0, 0, 0, 0, false};
        int k = sw;
        for (;; k += kSolveGroups) {
            locate(cur, blockIdx.x + k * (int)gridDim.x);
            if (!cur.valid) break;
            gbar_sync(3 + k % ns + ns * sw, kHandoff);  // group sw is done with unit k
            if (*(volatile int *)&s_stop) break;
            if (lane == 0) {
                int *sig[3] = {nullptr, nullptr, nullptr};
                if (cur.l < 0) {
                    sig[0] = done + (((cur.item * lv.coarse_rpu) / n2) << cl);
                } else {
                    const BcrItem it = items[lv.off[cur.l] + cur.item];
                    int *cnt_c = cnt + (size_t)cur.ch * sumK, *done_c = done + (size_t)cur.ch * sumK;
                    const int nr = n2 / cur.S, row0 = cur.sl * nr;
                    if (!phase_bwd(cur.ph)) {
                        if (it.right >= 0 && row0 + nr == n2) sig[0] = cnt_c + it.right;
                        if (it.left >= 0 && row0 == 0) sig[1] = cnt_c + it.left;
                        if (it.left < 0) sig[2] = done_c + it.cell;
                    } else {
                        sig[0] = done_c + it.cell;
                    }
                }
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (sig[q]) atomicAdd(sig[q], 1);
            }
            __syncwarp();
            // then the stage is refilled (the signal first: the dependency chain of the
            // narrow levels waits on it, the ring has n_stages - 1 other units in flight)
            locate(nxt, blockIdx.x + (k + ns) * (int)gridDim.x);
            if (nxt.valid) issue(nxt, k + ns);
        }
        // no copy may still be landing when the block exits: wait (bounded) for each
        // stage's latest fill (at once if it has landed; it is pending only after a stop)
        for (int st = 0; st < ns; ++st) {
            const int f = *(volatile int *)&s_fills[st];
            if (f > 0) tc::mbar_wait(&s_bar[st], (uint32_t)(f - 1) & 1u);
        }
        return;
    }
    // ---- compute groups
    const int grp = threadIdx.x / NTG;
    const Group gr{(int)threadIdx.x - grp * NTG, 1 + grp};
    T *smg = sm + grp * base;
    tc::grid_dependency_wait();  // the right-hand sides come from the previous kernel
    Pos cur{0, 0, 0, 0, 0, 0, 0, false};
    for (int k = grp;; k += kSolveGroups) {
        locate(cur, blockIdx.x + k * (int)gridDim.x);
        if (!cur.valid) break;
        const int st = k % ns;
        const uint32_t parity = (uint32_t)(k / ns) & 1u;
        T *As = stage_slice(st), *cb = stage_cpl(st);
        // bounded; a group whose copies never land records the error and stops (the
        // units left are then timed out by their consumers)
        auto wait_copies = [&]() {
            bool ok = true;
            if (*(volatile int *)&s_fills[st] <= k / ns) {  // the fill has not been issued yet
                const unsigned long long t0 = tc::global_ns();
                while (*(volatile int *)&s_fills[st] <= k / ns)
                    if (tc::global_ns() - t0 > tc::kWaitNs) {
                        ok = false;
                        break;
                    }
            }
            if (ok) ok = tc::mbar_wait(&s_bar[st], parity);
            const bool stalled = gbar_or(gr.bar, NTG, !ok);
            if (stalled && gr.gt == 0) {
                atomicExch(err, 1);
                s_stop = 1;
            }
            return !stalled;
        };
        bool ok;
        if (cur.l < 0) {
            // the stage's coupling area holds r_c (coarse units take no couplings)
            ok = ring_coarse_unit<T, NTG>(cur.item, lv, rhs, Y, N, cb, As, cnt, err, limit, gr, wait_copies);
        } else {
            const BcrItem it = items[lv.off[cur.l] + cur.item];
            const bool bwd = phase_bwd(cur.ph);
            const T *mB, *mC;
            unit_coupling_sources(it, cur.sl, cur.S, bwd, N, Bc, Cc, mB, mC);
            if (cb) {
                mB = mB ? cb : nullptr;
                mC = mC ? cb + hh : nullptr;
            }
            const int r0 = cur.ch * RC, nrc = min(RC, R - r0);
            const int *cnt_c = cnt + (size_t)cur.ch * sumK, *done_c = done + (size_t)cur.ch * sumK;
            FlowSync fs{};
            fs.err = err;
            fs.limit = limit;
            if (!bwd) {
                int want = 0;
                for (int lp = 0; lp < it.level; ++lp)
                    want += (it.local >= (1 << lp)) + (it.local + (1 << lp) < it.K_inst);
                if (want) {
                    fs.wait0 = cnt_c + it.cell;
                    fs.want0 = want;
                }
                ok = ring_fwd_unit<T, NTG, RC>(mB, mC, it, r0, nrc, cur.sl, cur.S, rhs, Y, N, sumK, smg, As,
                                               rhs_staged(cur, k) ? stage_rhs(st) : (const T *)nullptr, &fs, gr,
                                               wait_copies);
            } else {
                const int step = 1 << it.level;
                fs.wait0 = done_c + it.left;
                fs.want0 = done_want(bcr_cell_level(it.local - step, nl));
                if (it.right >= 0) {
                    fs.wait1 = done_c + it.right;
                    fs.want1 = done_want(bcr_cell_level(it.local + step, nl));
                }
                ok = ring_bwd_unit<T, NTG, RC>(mB, mC, it, r0, nrc, cur.sl, cur.S, Y, N, sumK, smg, As, &fs, gr,
                                               wait_copies);
            }
        }
        // every thread of the group has written and read what the unit needs before the handoff
        handoff_arrive(3 + st + ns * grp, kHandoff);
        if (!ok) break;
    }
}

// The inverse G of the coarse system (coarse_level c >= 0, one instance): the
// reduction's levels c .. n_levels - 1 and its root applied to the identity on the
// coarse cells' unknowns. Block b solves for the columns [b CB, (b + 1) CB): X (all
// coarse cells' 2N rows x CB columns, shared memory) starts as those identity
// columns; forward, each item of levels c .. up to the root replaces its X block by
// A^{-1} X and (below the root) pushes -B X[R+] into its right neighbour's L+ rows and
// -C X[L-] into its left neighbour's R- rows; backward, from the top level down, each
// item subtracts A^{-1}[:, L+ u R-] [B u_left[R+]; C u_right[L-]]. X then holds the
// columns of G (row-major, rows and columns in coarse order: cell-major, 2N per cell).
// Blocks that are still zero are skipped (forward, only the identity's cell and the
// cells it pushes into carry data). Each operation's A^{-1} columns and coupling
// blocks arrive in shared memory by bulk asynchronous copies (bounded waits; a block
// whose copies do not land records *err = 1 and stops).
template <typename T>
__host__ __device__ constexpr size_t coarse_inverse_values(int N, int m, int CB) {
    // X, g, A^{-1} columns, two coupling blocks (each area a whole number of 16-byte chunks)
    return ((size_t)m * 2 * N * CB + (size_t)N * CB + (size_t)4 * N * N + (size_t)2 * (N / 2) * (N / 2) +
            3 * 16 / sizeof(T));
}

template <typename T, int CB>
__global__ void __launch_bounds__(256) k_bcr_coarse_inverse(const T *__restrict__ A, const T *__restrict__ Bc,
                                                            const T *__restrict__ Cc,
                                                            const BcrItem *__restrict__ items, LevelTable lv, int N,
                                                            T *__restrict__ G, int *err) {
    static_assert(CB % 8 == 0, "8 columns per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const int n2 = 2 * N, h2 = N / 2, hh = h2 * h2, cl = lv.coarse_level, nl = lv.n_levels;
    const int m = lv.coarse_m, n = m * n2, j0 = blockIdx.x * CB;
    auto align16 = [](size_t v) { return (v * sizeof(T) + 15) / 16 * 16 / sizeof(T); };
    T *X = reinterpret_cast<T *>(smem_raw);  // [m][n2][CB]
    T *gs = X + align16((size_t)m * n2 * CB);  // [N][CB]
    T *F = gs + align16((size_t)N * CB);      // A^{-1} columns [k][n2]
    T *Cp = F + align16((size_t)n2 * n2);     // two coupling blocks [2][h2][h2]
    for (int idx = threadIdx.x; idx < n * CB; idx += blockDim.x) {
        const int row = idx / CB, col = idx - row * CB;
        X[idx] = (row == j0 + col) ? T(1) : T(0);
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // coarse cells holding nonzero data: bit j of nz (at most 64 coarse cells per word)
    unsigned long long nz[4] = {0ull, 0ull, 0ull, 0ull};
    auto get_nz = [&](int j) { return (nz[j >> 6] >> (j & 63)) & 1ull; };
    auto set_nz = [&](int j) { nz[j >> 6] |= 1ull << (j & 63); };
    for (int j = j0 / n2; j <= (j0 + CB - 1) / n2; ++j) set_nz(j);
    uint32_t parity = 0;
    bool ok = true;
    // copy A^{-1} columns [k0, k0 + nk) of cell and the coupling blocks m0, m1 (NULL: absent), then wait
    auto fetch = [&](int cell, int k0, int nk, const T *m0, const T *m1) {
        if (threadIdx.x == 0) {
            const uint32_t fb = (uint32_t)((size_t)nk * n2 * sizeof(T)), hb = (uint32_t)(hh * sizeof(T));
            tc::fence_async_smem();
            tc::mbar_arrive_expect_tx(&s_bar, fb + (m0 ? hb : 0u) + (m1 ? hb : 0u));
            tc::bulk_copy_g2s(F, A + (size_t)cell * n2 * n2 + (size_t)k0 * n2, fb, &s_bar);
            if (m0) tc::bulk_copy_g2s(Cp, m0, hb, &s_bar);
            if (m1) tc::bulk_copy_g2s(Cp + hh, m1, hb, &s_bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&s_bar, parity)) != 0;
        parity ^= 1u;
    };
    constexpr int CG = CB / 8;
    const int RT = blockDim.x / CG, r = threadIdx.x % RT, cgp = threadIdx.x / RT;
    // out (n2 x CB) (-)= F^T in: out[row] = sum_{kk < nk} F[kk][row] in[kk]
    auto apply = [&](int nk, const T *in, T *out, bool subtract) {
        T acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = T(0);
        if (r < n2) {
#pragma unroll 4
            for (int kk = 0; kk < nk; ++kk) {
                const T a = F[(size_t)kk * n2 + r];
                const T *x = in + (size_t)kk * CB + cgp * 8;
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = fma(a, x[c], acc[c]);
            }
        }
        __syncthreads();  // every read of in (possibly out) done
        if (r < n2) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                T *o = out + (size_t)r * CB + cgp * 8 + c;
                *o = subtract ? *o - acc[c] : acc[c];
            }
        }
        __syncthreads();
    };
    // out[p][c] (-)= sum_k M[p][k] v[k][c], p < h2 (M: h2 x h2 in shared memory)
    auto couple = [&](const T *M, const T *v, T *out, bool subtract) {
        for (int idx = threadIdx.x; idx < h2 * CB; idx += blockDim.x) {
            const int p = idx / CB, c = idx - p * CB;
            T s = T(0);
            for (int kk = 0; kk < h2; ++kk) s = fma(M[(size_t)p * h2 + kk], v[(size_t)kk * CB + c], s);
            out[(size_t)p * CB + c] = subtract ? out[(size_t)p * CB + c] - s : s;
        }
    };
    auto Xc = [&](int cell_local) { return X + (size_t)(cell_local >> cl) * n2 * CB; };
    for (int l = cl; l <= nl && ok; ++l) {
        const int i0 = lv.off[l], i1 = l < nl ? lv.off[l + 1] : lv.off[nl] + lv.n_roots;
        for (int ii = i0; ii < i1 && ok; ++ii) {
            const BcrItem it = items[ii];
            if (!get_nz(it.local >> cl)) continue;
            const int step = 1 << l;
            const bool pr = l < nl && it.right >= 0, pl = l < nl && it.left >= 0;
            fetch(it.cell, 0, n2, pr ? Bc + (size_t)it.s_right * hh : nullptr,
                  pl ? Cc + (size_t)it.s_left * hh : nullptr);
            if (!ok) break;
            T *Xi = Xc(it.local);
            apply(n2, Xi, Xi, false);
            if (pr) {
                couple(Cp, Xi + (size_t)(N + h2) * CB, Xc(it.local + step) + (size_t)h2 * CB, true);
                set_nz((it.local + step) >> cl);
            }
            if (pl) {
                couple(Cp + hh, Xi, Xc(it.local - step) + (size_t)N * CB, true);
                set_nz((it.local - step) >> cl);
            }
            __syncthreads();
        }
    }
    for (int l = nl - 1; l >= cl && ok; --l) {
        for (int ii = lv.off[l]; ii < lv.off[l + 1] && ok; ++ii) {
            const BcrItem it = items[ii];
            const int step = 1 << l, jl = (it.local - step) >> cl, jr = (it.local + step) >> cl;
            const bool rt = it.right >= 0;
            if (!get_nz(it.local >> cl) && !get_nz(jl) && !(rt && get_nz(jr))) continue;
            fetch(it.cell, h2, N, Bc + (size_t)it.s_cell * hh, rt ? Cc + (size_t)it.s_cell * hh : nullptr);
            if (!ok) break;
            couple(Cp, Xc(it.local - step) + (size_t)(N + h2) * CB, gs, false);
            if (rt) couple(Cp + hh, Xc(it.local + step), gs + (size_t)h2 * CB, false);
            else
                for (int idx = threadIdx.x; idx < h2 * CB; idx += blockDim.x) gs[(size_t)h2 * CB + idx] = T(0);
            __syncthreads();
            apply(N, gs, Xc(it.local), true);
            set_nz(it.local >> cl);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        tc::mbar_wait(&s_bar, parity ^ 1u);  // the copy that did not land in time (bounded)
        return;
    }
    for (int idx = threadIdx.x; idx < n * CB; idx += blockDim.x) {
        const int row = idx / CB, col = idx - row * CB;
        G[(size_t)row * n + j0 + col] = X[idx];
    }
}

// ---------------------------------------------------------------------------
// Adjoint (implicit differentiation of the converged discrete solution; the
// paper has no adjoint). The LD / S_N matrix A = L_h - S_h satisfies
// A^T = W Pi A Pi W^{-1} (W = diag(w_n) per node, Pi reverses the ordinates:
// the transposed upwind streaming of mu is the streaming of -mu, and S, the MPD
// and the WFD operators are w-self-adjoint and reversal-symmetric), so
// A^T lambda = s is solved as the forward system A x = Pi W^{-1} s with the
// same FPSA iteration and factors, lambda = W Pi x.
// Mirrored adjoint source as a nodal source of the sweep (b = m (x) q):
//   exit current (g == NULL): s_{K,R,n} = w_n mu_n for mu_n > 0, so
//     (Pi W^{-1} s) is |mu_n| at the last cell's right node for mu_n < 0;
//   moment functional <g, phi>: s = D^T g, so
//     (Pi W^{-1} s)_{a,n} = sum_l (-1)^l P_l(mu_n) g_{a,l}.
// q = m^{-1} (Pi W^{-1} s) per cell, m^{-1} = (2/h)[[2,-1],[-1,2]].
// Pm[n][l] = (-1)^l P_l(mu_n).
// ---------------------------------------------------------------------------
static __global__ void k_adjoint_source(const double *__restrict__ g, const double *__restrict__ Pm,
                                        const double *__restrict__ mu, const double *__restrict__ h,
                                        const int32_t *__restrict__ cell_inst, const int32_t *__restrict__ off,
                                        const int32_t *__restrict__ Kc, int N, int sumK, int R,
                                        double *__restrict__ q) {
    const size_t tot = (size_t)R * sumK * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(idx % N);
        const size_t rg = idx / N;  // r * sumK + cell
        const int cell = (int)(rg % sumK);
        double sL = 0.0, sR = 0.0;
        if (g) {
            const double *gL = g + (rg * 2) * N, *gR = gL + N;
            for (int l = 0; l < N; ++l) {
                const double p = Pm[(size_t)n * N + l];
                sL = fma(p, gL[l], sL);
                sR = fma(p, gR[l], sR);
            }
        } else {
            const int b = cell_inst[cell];
            if (cell == off[b] + Kc[b] - 1 && mu[n] < 0.0) sR = -mu[n];
        }
        const double w = 2.0 / h[cell];
        q[(rg * 2) * N + n] = w * (2.0 * sL - sR);
        q[(rg * 2 + 1) * N + n] = w * (2.0 * sR - sL);
    }
}

// Right-boundary exit current per (rhs, instance) from the forward moments:
// J = sum_{mu_n > 0} w_n mu_n psi_{K,R,n} = sum_l cJ[l] phi_{K,R,l}, cJ[l] =
// sum_{mu_n > 0} w_n mu_n (2l+1)/2 P_l(mu_n) (psi = M phi with all N moments).
static __global__ void k_exit_current(const double *__restrict__ phi, const double *__restrict__ cJ,
                                      const int32_t *__restrict__ off, const int32_t *__restrict__ Kc, int N,
                                      int sumK, int B, double *__restrict__ J) {
    const int b = blockIdx.x, r = blockIdx.y;
    const int cell = off[b] + Kc[b] - 1;
    const double *p = phi + (((size_t)r * sumK + cell) * 2 + 1) * N;
    double acc = 0.0;
    for (int l = threadIdx.x; l < N; l += 32) acc = fma(cJ[l], p[l], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) J[(size_t)r * B + b] = acc;
}

// Gradients from the forward moments phi and the mirrored adjoint moments x
// (both with all N moments), summed over right-hand sides:
//   t_l = (h/6) sum_r (2 x_L phi_L + x_L phi_R + x_R phi_L + 2 x_R phi_R)_l (2l+1)/2 (-1)^l
//   dJ/dsigma_s,l = t_l (l < L+1),   dJ/dsigma_t = -sum_{l<N} t_l
static __global__ void k_adjoint_grad(const double *__restrict__ phi, const double *__restrict__ x,
                                      const double *__restrict__ h, int N, int L1, int sumK, int R,
                                      double *__restrict__ d_st, double *__restrict__ d_ss) {
    __shared__ double red[32];
    const int g = blockIdx.x;
    double tsum = 0.0;
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
        double t = 0.0;
        for (int r = 0; r < R; ++r) {
            const size_t e = (((size_t)r * sumK + g) * 2) * N + l;
            const double xL = x[e], xR = x[e + N], pL = phi[e], pR = phi[e + N];
            t += 2.0 * xL * pL + xL * pR + xR * pL + 2.0 * xR * pR;
        }
        t *= h[g] / 6.0 * (l + 0.5) * ((l & 1) ? -1.0 : 1.0);
        if (l < L1) d_ss[(size_t)g * L1 + l] = t;
        tsum += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        d_st[g] = -s;
    }
}

}  // namespace fpsa
