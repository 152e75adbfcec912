// FMM matvec kernels (FP32) for the Helmholtz single-layer operator.
//
// One matvec (Sec. 2.3 and the Nystrom operator of Sec. 2.2):
//   density prep   sh_i = k w_i s_perm(i) / (4 pi)  (Morton order)
//   near field     phi_i  = sum_{j in direct leaves, j != i} sh_j (C(u)/sqrt(u) + i S(u)),
//                  u = (k R_ij)^2   [= w_j s_j exp(ikR)/(4 pi R), Eq. 6; Listing 1's P2P]
//   far field      P2M -> M2M -> M2L -> L2L -> L2P   (Eq. 11-14); an adaptive tree adds
//                  P2L after P2M and M2P after M2M for its W lists
//   correction     phi_i += sum_j C~_ij sh_j  (exact self/near integrals minus point terms)
//   output         potential[perm(i)] = phi_i
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <mutex>

#include "hfmm_internal.cuh"
#include "kernel_poly.h"

namespace hfmm {

// ============================================================== elementwise
template <typename T>
__global__ void k_density_prep(int64_t N, const int32_t* __restrict__ perm, const float* __restrict__ wscale,
                               const T* __restrict__ in, float2* __restrict__ sig) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T v = in[perm[i]];
    float w = wscale[i];
    sig[i] = make_float2(w * (float)v.x, w * (float)v.y);
}

template <typename T>
__global__ void k_output(int64_t N, const int32_t* __restrict__ perm, const float2* __restrict__ phi,
                         T* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float2 v = phi[i];
    T o{};  // a double-float output (float4) gets zero low parts
    o.x = v.x;
    o.y = v.y;
    out[perm[i]] = o;
}

void launch_density_prep(hfmm_plan* P, const void* density, VecKind kind, float2* sig, cudaStream_t st) {
    ++P->launches;
    unsigned nb = (unsigned)((P->N + 255) / 256);
    if (kind == VecKind::DoubleFloat)  // (re_hi, im_hi, re_lo, im_lo): the FP32 value is the high part
        k_density_prep<float4><<<nb, 256, 0, st>>>(P->N, P->perm.p, P->wscale.p, (const float4*)density, sig);
    else
        k_density_prep<float2><<<nb, 256, 0, st>>>(P->N, P->perm.p, P->wscale.p, (const float2*)density, sig);
}

void launch_output(hfmm_plan* P, const float2* phi, void* out, VecKind kind, cudaStream_t st) {
    ++P->launches;
    unsigned nb = (unsigned)((P->N + 255) / 256);
    if (kind == VecKind::DoubleFloat) k_output<float4><<<nb, 256, 0, st>>>(P->N, P->perm.p, phi, (float4*)out);
    else k_output<float2><<<nb, 256, 0, st>>>(P->N, P->perm.p, phi, (float2*)out);
}

// ============================================================== near field (P2P)
template <int D>
__device__ __forceinline__ float horner(const float (&c)[D + 1], float u) {
    float a = c[D];
#pragma unroll
    for (int q = D - 1; q >= 0; --q) a = fmaf(a, u, c[q]);
    return a;
}

// Accumulates the interactions of one target with the points j0, j0+stride, ... < j1
// of one source leaf.  (tx,ty,tz): target relative to the source leaf centre, scaled by k.
template <bool POLY, bool MASK>
__device__ __forceinline__ void p2p_leaf(float tx, float ty, float tz, int32_t j0, int32_t j1, int32_t self_i,
                                         const float4* __restrict__ pts, const float2* __restrict__ sig,
                                         float& ar, float& ai) {
    constexpr float kC[HFMM_POLY_C_DEG + 1] = HFMM_POLY_C_INIT;
    constexpr float kS[HFMM_POLY_S_DEG + 1] = HFMM_POLY_S_INIT;
#pragma unroll 4
    for (int32_t j = j0; j < j1; j += kP2PSub) {
        float4 sp = __ldg(pts + j);
        float2 sg = __ldg(sig + j);
        if (MASK && j == self_i) sg = make_float2(0.f, 0.f);
        float dx = tx - sp.x, dy = ty - sp.y, dz = tz - sp.z;
        float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float rinv = rsqrtf(fmaxf(u, 1e-30f));
        float re, im;
        if (POLY) {
            re = horner<HFMM_POLY_C_DEG>(kC, u) * rinv;  // cos(kR)/(kR)
            im = horner<HFMM_POLY_S_DEG>(kS, u);         // sin(kR)/(kR)
        } else {
            float r = u * rinv, sn, cs;
            sincosf(r, &sn, &cs);
            re = cs * rinv;
            im = sn * rinv;
        }
        ar = fmaf(sg.x, re, fmaf(-sg.y, im, ar));
        ai = fmaf(sg.x, im, fmaf(sg.y, re, ai));
    }
}

// One warp per tile of up to kP2PTile targets of one leaf; each target is
// shared by kP2PSub lanes that take every kP2PSub-th source, and the partial
// sums meet in two shuffles.  Source loads are broadcast within each group of
// lanes that read the same point.
template <bool POLY>
__global__ void __launch_bounds__(256) k_p2p(int64_t ntiles, const int4* __restrict__ tiles,
                                             const int32_t* __restrict__ leaf_start,
                                             const int4* __restrict__ leaf_ijk,
                                             const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr,
                                             const float4* __restrict__ pts, const float2* __restrict__ sig,
                                             float shift, float2* __restrict__ phi) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= ntiles) return;
    int4 tl = tiles[w];
    int leaf = tl.x;
    const int tloc = lane / kP2PSub, sub = lane % kP2PSub;
    bool active = tloc < tl.z;
    int32_t i = tl.y + (active ? tloc : 0);
    float4 t = __ldg(pts + i);
    int4 tij = __ldg(leaf_ijk + leaf);
    float ar = 0.f, ai = 0.f;
    int32_t nb0 = nbr_ptr[leaf], nb1 = nbr_ptr[leaf + 1];
    for (int32_t q = nb0; q < nb1; ++q) {
        int32_t s = __ldg(nbr + q);
        int4 sij = __ldg(leaf_ijk + s);
        float tx = fmaf((float)(tij.x - sij.x), shift, t.x);
        float ty = fmaf((float)(tij.y - sij.y), shift, t.y);
        float tz = fmaf((float)(tij.z - sij.z), shift, t.z);
        int32_t j0 = __ldg(leaf_start + s) + sub, j1 = __ldg(leaf_start + s + 1);
        if (s == leaf) p2p_leaf<POLY, true>(tx, ty, tz, j0, j1, i, pts, sig, ar, ai);
        else p2p_leaf<POLY, false>(tx, ty, tz, j0, j1, i, pts, sig, ar, ai);
    }
#pragma unroll
    for (int o = 1; o < kP2PSub; o <<= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (active && sub == 0) phi[i] = make_float2(ar, ai);
}

// One block (4 warps) per target leaf.  The sources of all neighbour leaves are
// staged once in shared memory, shifted into the target leaf's frame, self leaf
// first (its entries are the targets themselves).  Warp w handles target tiles
// w, w+4, ...; within a tile each target is shared by kP2PSub lanes.  The self
// segment carries the j != i mask and the u = 0 guard; the rest runs unmasked.
// hardware reciprocal square root; its inputs are normal numbers (distinct points, or the guard)
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool POLY, bool MASK>
__device__ __forceinline__ void p2p_span(float tx, float ty, float tz, int k0, int k1, int self_k,
                                         const float4* __restrict__ sp, const float* __restrict__ sim,
                                         float& ar, float& ai) {
    constexpr float kC[HFMM_POLY_C_DEG + 1] = HFMM_POLY_C_INIT;
    constexpr float kS[HFMM_POLY_S_DEG + 1] = HFMM_POLY_S_INIT;
#pragma unroll 4
    for (int k = k0; k < k1; k += kP2PSub) {
        const float4 q = sp[k];  // x, y, z, Re sigma
        float sr = q.w, si = sim[k];
        if (MASK && k == self_k) sr = si = 0.f;
        const float dx = tx - q.x, dy = ty - q.y, dz = tz - q.z;
        const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrt_ftz(MASK ? fmaxf(u, 1e-30f) : u);
        float re, im;
        if (POLY) {
            re = horner<HFMM_POLY_C_DEG>(kC, u) * rinv;
            im = horner<HFMM_POLY_S_DEG>(kS, u);
        } else {
            float r = u * rinv, sn, cs;
            sincosf(r, &sn, &cs);
            re = cs * rinv;
            im = sn * rinv;
        }
        ar = fmaf(sr, re, fmaf(-si, im, ar));
        ai = fmaf(sr, im, fmaf(si, re, ai));
    }
}

constexpr int kStagedNbr = 64;  // most source leaves the staged kernel takes (27 in a uniform tree)

// Neighbourhood table of target leaf b for the staged near-field kernels, built by one warp
// in parallel (one neighbour per lane, counts prefix-summed with shuffles): entry q names
// the first point s_j0[q] and count s_cnt[q] of source leaf q (q = 0: the target leaf
// itself), its first staged index s_off[q] and the shift s_sh[q] of its frame into b's.
// pad: the self segment and the total are rounded up to even lengths.  *s_nl = entries;
// s_off[*s_nl] = total.
struct NbrTable {
    int off[kStagedNbr + 1], j0[kStagedNbr], cnt[kStagedNbr], nl;
    float4 sh[kStagedNbr];
};

__device__ void build_nbr_table(int b, const int32_t* __restrict__ leaf_start, const int4* __restrict__ leaf_ijk,
                                const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr, float shift,
                                bool pad, NbrTable& T) {
    const int lane = threadIdx.x & 31;
    const int nb0 = __ldg(nbr_ptr + b), nn = __ldg(nbr_ptr + b + 1) - nb0;
    const int4 tij = __ldg(leaf_ijk + b);
    const int j0b = __ldg(leaf_start + b), nself = __ldg(leaf_start + b + 1) - j0b;
    if (lane == 0) {
        T.j0[0] = j0b;
        T.cnt[0] = nself;
        T.off[0] = 0;
        T.sh[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int base = pad ? ((nself + 1) & ~1) : nself, k = 1;
    for (int q0 = 0; q0 < nn; q0 += 32) {
        const int q = q0 + lane;
        int sl = -1, cnt = 0, j0 = 0;
        if (q < nn) {
            sl = __ldg(nbr + nb0 + q);
            if (sl == b) sl = -1;
        }
        if (sl >= 0) {
            j0 = __ldg(leaf_start + sl);
            cnt = __ldg(leaf_start + sl + 1) - j0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, sl >= 0);
        int x = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        const int slot = k + __popc(m & ((1u << lane) - 1u));
        if (sl >= 0 && slot < kStagedNbr) {
            const int4 sij = __ldg(leaf_ijk + sl);
            T.j0[slot] = j0;
            T.cnt[slot] = cnt;
            T.off[slot] = base + x - cnt;
            T.sh[slot] = make_float4((float)(sij.x - tij.x) * shift, (float)(sij.y - tij.y) * shift,
                                     (float)(sij.z - tij.z) * shift, 0.f);
        }
        base += __shfl_sync(0xffffffffu, x, 31);
        k += __popc(m);
    }
    if (lane == 0) {
        T.off[k] = pad ? ((base + 1) & ~1) : base;
        T.nl = k;
    }
}

// segment q of staged index p: the last q with T.off[q] <= p
__device__ __forceinline__ int nbr_segment(const NbrTable& T, int p) {
    int lo = 0, hi = T.nl;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (T.off[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}
template <bool POLY>
__global__ void __launch_bounds__(128) k_p2p_staged(const int32_t* __restrict__ leaf_start,
                                                    const int4* __restrict__ leaf_ijk,
                                                    const int32_t* __restrict__ nbr_ptr,
                                                    const int32_t* __restrict__ nbr,
                                                    const float4* __restrict__ pts,
                                                    const float2* __restrict__ sig, float shift, int cap,
                                                    float2* __restrict__ phi) {
    extern __shared__ float4 sp[];  // [cap]: shifted position, Re sigma
    float* sim = reinterpret_cast<float*>(sp + cap);  // [cap]: Im sigma
    __shared__ NbrTable T;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tid < 32) build_nbr_table(b, leaf_start, leaf_ijk, nbr_ptr, nbr, shift, false, T);
    __syncthreads();
    const int total = T.off[T.nl];
    for (int p = tid; p < total; p += blockDim.x) {  // one flat pass: loads of all leaves in flight
        const int q = nbr_segment(T, p);
        const int e = p - T.off[q];
        const float4 pt = __ldg(pts + T.j0[q] + e);
        const float2 g = __ldg(sig + T.j0[q] + e);
        const float4 o = T.sh[q];
        sp[p] = make_float4(pt.x + o.x, pt.y + o.y, pt.z + o.z, g.x);
        sim[p] = g.y;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int nself = T.cnt[0];
    const int tloc = lane / kP2PSub, sub = lane % kP2PSub;
    for (int tile = warp; tile * kP2PTile < nself; tile += 4) {
        const int it = tile * kP2PTile + tloc;
        const bool active = it < nself;
        const int ik = active ? it : 0;
        const float4 t = sp[ik];
        float ar = 0.f, ai = 0.f;
        p2p_span<POLY, true>(t.x, t.y, t.z, sub, nself, ik, sp, sim, ar, ai);
        p2p_span<POLY, false>(t.x, t.y, t.z, nself + sub, total, -1, sp, sim, ar, ai);
#pragma unroll
        for (int o = 1; o < kP2PSub; o <<= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (active && sub == 0) phi[__ldg(leaf_start + b) + it] = make_float2(ar, ai);
    }
}

// ------------------------------------------------------------------ packed near field
// One block per target leaf.  The neighbourhood's sources are staged in shared memory in
// pairs, laid out so that each operand of a pair is an aligned register pair:
//   sq[2q]   = {x_2q, x_2q+1, y_2q, y_2q+1},  sq[2q+1] = {z_2q, z_2q+1, Re s_2q, Re s_2q+1},
//   sim[q]   = {Im s_2q, Im s_2q+1}
// (self leaf first, each of the two segments padded to an even length with a zero-density
// source far away).  A thread holds kPkTargets targets and evaluates both sources of a pair
// at once for each of them with packed FP32x2 arithmetic (fma.rn.f32x2 and friends), walking
// every S-th pair; the S threads that share a target meet in shared memory.  The complex multiply-add is kept as
// four real accumulators (Re s Re G, Im s Im G, Re s Im G, Im s Re G), so it needs no
// negated operand.  Same kernel (cos, sinc polynomials in u = (kR)^2, hardware rsqrt) and
// the same j != i rule as the staged kernel above.
constexpr int kPkThreads = 128;
constexpr int kPkTargets = 2;  // targets per thread
constexpr float kPkPad = 64.0f;  // padding sources sit at (64, 64, 64) (scaled units): u stays finite

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

template <int D>
__device__ __forceinline__ float2 horner2(const float (&c)[D + 1], float2 u) {
    float2 a = f2(c[D]);
#pragma unroll
    for (int q = D - 1; q >= 0; --q) a = __ffma2_rn(a, u, f2(c[q]));
    return a;
}

// d2 = 2q - (target's staged index): half 0 of the pair is the target itself when d2 == 0,
// half 1 when d2 == -1 (MASK: the self segment only)
template <bool MASK>
__device__ __forceinline__ void pk_pair(const float4 xy, const float4 zr, float2 si, float2 ntx, float2 nty, float2 ntz,
                                        int d2, float2& A, float2& B, float2& C, float2& D) {
    constexpr float kC[HFMM_POLY_C_DEG + 1] = HFMM_POLY_C_INIT;
    constexpr float kS[HFMM_POLY_S_DEG + 1] = HFMM_POLY_S_INIT;
    const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), ntx);
    const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), nty);
    const float2 dz = __fadd2_rn(make_float2(zr.x, zr.y), ntz);
    float2 u = __fmul2_rn(dz, dz);
    u = __ffma2_rn(dy, dy, u);
    u = __ffma2_rn(dx, dx, u);
    float2 sr = make_float2(zr.z, zr.w);
    if (MASK) {
        if (d2 == 0) sr.x = si.x = 0.f;
        if (d2 == -1) sr.y = si.y = 0.f;
        u.x = fmaxf(u.x, 1e-30f);
        u.y = fmaxf(u.y, 1e-30f);
    }
    const float2 rinv = make_float2(rsqrt_ftz(u.x), rsqrt_ftz(u.y));
    const float2 re = __fmul2_rn(horner2<HFMM_POLY_C_DEG>(kC, u), rinv);  // cos(kR)/(kR)
    const float2 im = horner2<HFMM_POLY_S_DEG>(kS, u);                     // sin(kR)/(kR)
    A = __ffma2_rn(sr, re, A);
    B = __ffma2_rn(si, im, B);
    C = __ffma2_rn(sr, im, C);
    D = __ffma2_rn(si, re, D);
}

// ten blocks per SM (48 registers): measured faster than the unconstrained 64
template <int TPT>
__global__ void __launch_bounds__(kPkThreads, 10) k_p2p_packed(const int32_t* __restrict__ leaf_start,
                                                           const int4* __restrict__ leaf_ijk,
                                                           const int32_t* __restrict__ nbr_ptr,
                                                           const int32_t* __restrict__ nbr,
                                                           const float4* __restrict__ pts,
                                                           const float2* __restrict__ sig, float shift, int cap_pairs,
                                                           float2* __restrict__ phi) {
    extern __shared__ float4 sq[];                                   // [2 cap_pairs]
    float2* sim = reinterpret_cast<float2*>(sq + 2 * cap_pairs);    // [cap_pairs]
    __shared__ NbrTable T;
    __shared__ float2 s_red[TPT][kPkThreads];
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tid < 32) build_nbr_table(b, leaf_start, leaf_ijk, nbr_ptr, nbr, shift, true, T);
    __syncthreads();
    const int total = T.off[T.nl], npair = total >> 1;
    const int nself = T.cnt[0];
    const int qself = T.off[1] >> 1;  // pairs of the self segment (padded to even)
    float* sf = reinterpret_cast<float*>(sq);
    float* sfi = reinterpret_cast<float*>(sim);
    for (int p = tid; p < total; p += kPkThreads) {  // one flat pass: loads of all leaves in flight
        const int q = nbr_segment(T, p);
        const int e = p - T.off[q];
        float x = kPkPad, y = kPkPad, z = kPkPad, sr = 0.f, si = 0.f;
        if (e < T.cnt[q]) {
            const float4 pt = __ldg(pts + T.j0[q] + e);
            const float2 g = __ldg(sig + T.j0[q] + e);
            const float4 o = T.sh[q];
            x = pt.x + o.x;
            y = pt.y + o.y;
            z = pt.z + o.z;
            sr = g.x;
            si = g.y;
        }
        const int pq = p >> 1, h = p & 1;
        float* r = sf + 8 * pq;
        r[h] = x;
        r[2 + h] = y;
        r[4 + h] = z;
        r[6 + h] = sr;
        sfi[2 * pq + h] = si;
    }
    __syncthreads();
    // TPT targets per thread (slot, slot + TT, ...): every source pair read from shared memory
    // serves all of them, so the loads and the loop's index work are shared
    const int TT = min((nself + TPT - 1) / TPT, kPkThreads);  // target slots per round
    const int S = kPkThreads / max(TT, 1);                     // threads sharing a slot
    const int slot = tid % max(TT, 1), sp = tid / max(TT, 1);
    const int i0 = __ldg(leaf_start + b);
    for (int t0 = 0; t0 < nself; t0 += TT * TPT) {
        int it[TPT];
        float ar[TPT], ai[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            it[k] = t0 + slot + k * TT;
            ar[k] = ai[k] = 0.f;
        }
        if (sp < S && it[0] < nself) {
            float2 ntx[TPT], nty[TPT], ntz[TPT], A[TPT], B[TPT], C[TPT], D[TPT];
            int ik[TPT];  // staged index of each target (a missing one repeats the first)
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                ik[k] = it[k] < nself ? it[k] : it[0];
                const float* tr = sf + 8 * (ik[k] >> 1) + (ik[k] & 1);
                ntx[k] = f2(-tr[0]);
                nty[k] = f2(-tr[2]);
                ntz[k] = f2(-tr[4]);
                A[k] = B[k] = C[k] = D[k] = f2(0.f);
            }
            int q = sp;
            for (; q < qself; q += S) {
                const float4 xy = sq[2 * q], zr = sq[2 * q + 1];
                const float2 si = sim[q];
#pragma unroll
                for (int k = 0; k < TPT; ++k)
                    pk_pair<true>(xy, zr, si, ntx[k], nty[k], ntz[k], 2 * q - ik[k], A[k], B[k], C[k], D[k]);
            }
#pragma unroll 1  // rolled: unrolling by 2 or 4 measured slower
            for (; q < npair; q += S) {
                const float4 xy = sq[2 * q], zr = sq[2 * q + 1];
                const float2 si = sim[q];
#pragma unroll
                for (int k = 0; k < TPT; ++k)
                    pk_pair<false>(xy, zr, si, ntx[k], nty[k], ntz[k], 0, A[k], B[k], C[k], D[k]);
            }
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                ar[k] = (A[k].x + A[k].y) - (B[k].x + B[k].y);
                ai[k] = (C[k].x + C[k].y) + (D[k].x + D[k].y);
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; ++k) s_red[k][tid] = make_float2(ar[k], ai[k]);
        __syncthreads();
        if (sp == 0) {
#pragma unroll
            for (int k = 0; k < TPT; ++k)
                if (it[k] < nself) {
                    float2 acc = s_red[k][slot];
                    for (int r = 1; r < S; ++r) {
                        const float2 v = s_red[k][slot + r * TT];
                        acc.x += v.x;
                        acc.y += v.y;
                    }
                    phi[i0 + it[k]] = acc;
                }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ pipelined near field
// The packed kernel's arithmetic in persistent blocks that walk leaves b, b + grid, ...: while
// a block evaluates one leaf, the next leaf's sources travel from global to shared memory with
// cp.async (raw, as stored), so the global loads no longer sit in front of a block barrier;
// after the evaluation they are shifted into the leaf's frame and laid out in pairs from shared
// memory.  Same pairs, the same per-pair arithmetic and the same j != i rule as k_p2p_packed.
constexpr int kPipeBlocksPerSM = 8;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__global__ void __launch_bounds__(kPkThreads) k_p2p_pipe(int nleaf, const int32_t* __restrict__ leaf_start,
                                                         const int4* __restrict__ leaf_ijk,
                                                         const int32_t* __restrict__ nbr_ptr,
                                                         const int32_t* __restrict__ nbr,
                                                         const float4* __restrict__ pts,
                                                         const float2* __restrict__ sig, float shift, int cap_pairs,
                                                         float2* __restrict__ phi) {
    extern __shared__ float4 sq[];                                  // [2 cap_pairs] pairs (packed layout)
    float4* rawp = sq + 2 * cap_pairs;                              // [2 cap_pairs] next leaf's positions
    float2* sim = reinterpret_cast<float2*>(rawp + 2 * cap_pairs);  // [cap_pairs]
    float2* raws = sim + cap_pairs;                                 // [2 cap_pairs] next leaf's densities
    __shared__ NbrTable TT[2];
    __shared__ float2 s_red[kPkThreads];
    const int tid = threadIdx.x;
    float* sf = reinterpret_cast<float*>(sq);
    float* sfi = reinterpret_cast<float*>(sim);
    auto issue = [&](const NbrTable& T) {  // raw copies of the neighbourhood, padding slots left out
        const int total = T.off[T.nl];
        for (int p = tid; p < total; p += kPkThreads) {
            const int q = nbr_segment(T, p);
            const int e = p - T.off[q];
            if (e < T.cnt[q]) {
                cp_async16(rawp + p, pts + T.j0[q] + e);
                cp_async8(raws + p, sig + T.j0[q] + e);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto pack = [&](const NbrTable& T) {  // raw -> shifted pairs (padding: far away, zero density)
        const int total = T.off[T.nl];
        for (int p = tid; p < total; p += kPkThreads) {
            const int q = nbr_segment(T, p);
            const int e = p - T.off[q];
            float x = kPkPad, y = kPkPad, z = kPkPad, sr = 0.f, si = 0.f;
            if (e < T.cnt[q]) {
                const float4 pt = rawp[p];
                const float2 g = raws[p];
                const float4 o = T.sh[q];
                x = pt.x + o.x;
                y = pt.y + o.y;
                z = pt.z + o.z;
                sr = g.x;
                si = g.y;
            }
            const int pq = p >> 1, h = p & 1;
            float* r = sf + 8 * pq;
            r[h] = x;
            r[2 + h] = y;
            r[4 + h] = z;
            r[6 + h] = sr;
            sfi[2 * pq + h] = si;
        }
    };
    int b = blockIdx.x;
    if (b >= nleaf) return;  // uniform over the block
    int cur = 0;
    if (tid < 32) build_nbr_table(b, leaf_start, leaf_ijk, nbr_ptr, nbr, shift, true, TT[0]);
    __syncthreads();
    issue(TT[0]);
    cp_async_wait_all();
    __syncthreads();
    pack(TT[0]);
    __syncthreads();
    for (; b < nleaf; b += gridDim.x) {
        const int bn = b + gridDim.x;
        const bool more = bn < nleaf;  // uniform over the block
        if (more) {
            if (tid < 32) build_nbr_table(bn, leaf_start, leaf_ijk, nbr_ptr, nbr, shift, true, TT[cur ^ 1]);
            __syncthreads();
            issue(TT[cur ^ 1]);
        }
        const NbrTable& T = TT[cur];
        const int npair = T.off[T.nl] >> 1;
        const int nself = T.cnt[0];
        const int qself = T.off[1] >> 1;
        const int TTn = min(nself, kPkThreads);
        const int S = kPkThreads / max(TTn, 1);
        const int slot = tid % max(TTn, 1), sp = tid / max(TTn, 1);
        const int i0 = __ldg(leaf_start + b);
        for (int t0 = 0; t0 < nself; t0 += TTn) {
            const int it = t0 + slot;
            float ar = 0.f, ai = 0.f;
            if (sp < S && it < nself) {
                const float* tr = sf + 8 * (it >> 1) + (it & 1);
                const float2 ntx = f2(-tr[0]), nty = f2(-tr[2]), ntz = f2(-tr[4]);
                float2 A = f2(0.f), B = f2(0.f), C = f2(0.f), D = f2(0.f);
                int q = sp;
                for (; q < qself; q += S)
                    pk_pair<true>(sq[2 * q], sq[2 * q + 1], sim[q], ntx, nty, ntz, 2 * q - it, A, B, C, D);
#pragma unroll 2
                for (; q < npair; q += S) pk_pair<false>(sq[2 * q], sq[2 * q + 1], sim[q], ntx, nty, ntz, 0, A, B, C, D);
                ar = (A.x + A.y) - (B.x + B.y);
                ai = (C.x + C.y) + (D.x + D.y);
            }
            s_red[tid] = make_float2(ar, ai);
            __syncthreads();
            if (sp == 0 && it < nself) {
                float2 acc = s_red[slot];
                for (int r = 1; r < S; ++r) {
                    const float2 v = s_red[slot + r * TTn];
                    acc.x += v.x;
                    acc.y += v.y;
                }
                phi[i0 + it] = acc;
            }
            __syncthreads();
        }
        if (more) {
            cp_async_wait_all();  // this thread's copies of the next leaf
            __syncthreads();      // everyone's, and the pairs of this leaf are no longer read
            pack(TT[cur ^ 1]);
            __syncthreads();
            cur ^= 1;
        }
    }
}

// ============================================================== FP32 special functions
// out[n] = j_n(x) / s^n, n = 0..p
// Reciprocals for the small-argument series of j_n (uploaded with the Legendre tables):
// c_jser[n][q] = 1 / (q (2n + 2q + 1)), c_inv_odd[n] = 1 / (2n + 1).
constexpr int kJTerms = 24;
__constant__ float c_jser[HFMM_PMAX + 1][kJTerms];
__constant__ float c_inv_odd[HFMM_PMAX + 1];

// j_n(x) / s^n for x < 2: (x/s)^n / (2n+1)!! * sum_q prod_{i<=q} (-x^2/2) / (i (2n+2i+1))
__device__ __forceinline__ float f_jn_series(int n, float x, float s) {
    float lead = 1.0f;
    const float xs = x / s, h = -0.5f * x * x;
    for (int i = 1; i <= n; ++i) lead *= xs * c_inv_odd[i];
    float term = 1.0f, sum = 1.0f;
    for (int q = 1; q < kJTerms; ++q) {
        term *= h * c_jser[n][q];
        sum += term;
        if (fabsf(term) < 1e-8f * fabsf(sum)) break;
    }
    return lead * sum;
}

__device__ static void f_jn_scaled(int p, float x, float s, float* out) {
    if (x < 2.0f) {
        for (int n = 0; n <= p; ++n) out[n] = f_jn_series(n, x, s);
        return;
    }
    int top = p + 16 + (int)x;
    float fn1 = 0.f, fn = 1e-20f;
    for (int n = top; n > p; --n) {
        float f = (float)(2 * n + 1) / x * fn - fn1;
        fn1 = fn;
        fn = f;
        if (fabsf(fn) > 1e20f) { fn *= 1e-20f; fn1 *= 1e-20f; }
    }
    out[p] = fn;
    float up = fn1;
    for (int n = p; n >= 1; --n) {
        float f = (float)(2 * n + 1) / x * out[n] - up;
        up = out[n];
        out[n - 1] = f;
        if (fabsf(f) > 1e20f) {
            for (int m = n - 1; m <= p; ++m) out[m] *= 1e-20f;
            up *= 1e-20f;
        }
    }
    float sx, cx;
    sincosf(x, &sx, &cx);
    float j0 = sx / x, j1 = sx / (x * x) - cx / x;
    float c = fabsf(j0) > fabsf(j1) ? j0 / out[0] : j1 / out[1];
    float sp = 1.f;
    for (int n = 0; n <= p; ++n) {
        out[n] *= c / sp;
        sp *= s;
    }
}

struct Dir {
    float ct, st, ex, ey, r;
};
__device__ __forceinline__ Dir make_dir(float x, float y, float z) {
    Dir d;
    float r2 = x * x + y * y + z * z;
    d.r = sqrtf(r2);
    d.ct = 1.f;
    d.st = 0.f;
    d.ex = 1.f;
    d.ey = 0.f;
    if (d.r > 0.f) {
        d.ct = z / d.r;
        float rxy = sqrtf(x * x + y * y);
        d.st = rxy / d.r;
        if (rxy > 0.f) {
            d.ex = x / rxy;
            d.ey = y / rxy;
        }
    }
    return d;
}

// ============================================================== Legendre tables
// Normalised associated Legendre functions Q_n^m (orthonormal Y without the
// Condon-Shortley phase):  Q_m^m = qmm[m] sin^m,  Q_{m+1}^m = sqrt(2m+3) cos Q_m^m,
// Q_n^m = a_nm (cos Q_{n-1}^m - b_nm Q_{n-2}^m), indexed by n(n+1)/2 + m.
constexpr int kLegH = (HFMM_PMAX + 1) * (HFMM_PMAX + 2) / 2;
__constant__ float c_leg_a[kLegH];
__constant__ float c_leg_b[kLegH];
__constant__ float c_leg_qmm[HFMM_PMAX + 1];

void upload_legendre_tables() {
    static bool done[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return;
    std::vector<float> a(kLegH, 0.f), b(kLegH, 0.f), q(HFMM_PMAX + 1, 0.f);
    double qmm = 0.28209479177387814;  // 1/sqrt(4 pi)
    for (int m = 0; m <= HFMM_PMAX; ++m) {
        if (m > 0) qmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m));
        q[m] = (float)qmm;
        for (int n = m; n <= HFMM_PMAX; ++n) {
            int h = n * (n + 1) / 2 + m;
            if (n == m + 1) a[h] = (float)std::sqrt(2.0 * m + 3.0);
            if (n >= m + 2) {
                a[h] = (float)std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
                b[h] = (float)std::sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
            }
        }
    }
    HFMM_CUDA(cudaMemcpyToSymbol(c_leg_a, a.data(), sizeof(float) * kLegH));
    HFMM_CUDA(cudaMemcpyToSymbol(c_leg_b, b.data(), sizeof(float) * kLegH));
    HFMM_CUDA(cudaMemcpyToSymbol(c_leg_qmm, q.data(), sizeof(float) * (HFMM_PMAX + 1)));
    std::vector<float> js((HFMM_PMAX + 1) * kJTerms, 0.f), io(HFMM_PMAX + 1, 0.f);
    for (int n = 0; n <= HFMM_PMAX; ++n) {
        io[n] = (float)(1.0 / (2.0 * n + 1.0));
        for (int t = 1; t < kJTerms; ++t) js[n * kJTerms + t] = (float)(1.0 / ((double)t * (2.0 * n + 2.0 * t + 1.0)));
    }
    HFMM_CUDA(cudaMemcpyToSymbol(c_jser, js.data(), sizeof(float) * js.size()));
    HFMM_CUDA(cudaMemcpyToSymbol(c_inv_odd, io.data(), sizeof(float) * io.size()));
    if (dev < 64) done[dev] = true;
}

// ============================================================== P2M
// One block (128 threads) per leaf; points are taken in chunks of up to 32:
//   phase 1: thread j computes the scaled radial functions jt_n(k r_j), n <= p;
//   phase 2: thread (m, j) runs the Legendre recurrence in n for its order m and
//            stores jt_n Q_n^m and sh e^{-/+ i m phi};
//   phase 3: thread c accumulates coefficient c = n^2 + n + m over the chunk.
__global__ void __launch_bounds__(128) k_p2m(const int32_t* __restrict__ leaf_start,
                                             const float4* __restrict__ pts, const float2* __restrict__ sig,
                                             int p, float s, float2* __restrict__ M,
                                             const int32_t* __restrict__ leaf_lev, int lev,
                                             const int32_t* __restrict__ leaf_box) {
    constexpr int kChunk = 32;
    extern __shared__ float sm[];
    const int leaf = blockIdx.x;
    if (leaf_lev && leaf_lev[leaf] != lev) return;  // uniform over the block: before any barrier
    const int64_t box = leaf_box ? leaf_box[leaf] : leaf;
    const int P = (p + 1) * (p + 1);
    const int H = (p + 1) * (p + 2) / 2;
    float* rad = sm;                          // [kChunk][p+1]
    float* B = rad + kChunk * (p + 1);        // [kChunk][H]
    float* E = B + kChunk * H;                // [kChunk][p+1][4]
    float* geo = E + kChunk * (p + 1) * 4;    // [kChunk][4]: cos t, sin t, cos phi, sin phi
    float* rr = geo + kChunk * 4;             // [kChunk]: k r
    const int32_t b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    // two coefficients per thread per pass; orders above 14 take more passes
    for (int cg = 0; cg < P; cg += 256) {
        int cc[2], hidx[2], eo[2];
        for (int q = 0; q < 2; ++q) {
            cc[q] = cg + threadIdx.x + 128 * q;
            int n = 0, m = 0;
            if (cc[q] < P) {
                n = (int)sqrtf((float)cc[q]);
                while (n * n > cc[q]) --n;
                while ((n + 1) * (n + 1) <= cc[q]) ++n;
                m = cc[q] - n * n - n;
            }
            hidx[q] = n * (n + 1) / 2 + (m < 0 ? -m : m);
            eo[q] = 4 * (m < 0 ? -m : m) + (m < 0 ? 2 : 0);
        }
        float accr[2] = {0.f, 0.f}, acci[2] = {0.f, 0.f};
        for (int32_t j0 = b0; j0 < b1; j0 += kChunk) {
            const int cnt = min(kChunk, b1 - j0);
            if (threadIdx.x < cnt) {
                const int j = threadIdx.x;
                const float4 y = pts[j0 + j];
                const Dir d = make_dir(y.x, y.y, y.z);
                geo[4 * j + 0] = d.ct;
                geo[4 * j + 1] = d.st;
                geo[4 * j + 2] = d.ex;
                geo[4 * j + 3] = d.ey;
                rr[j] = d.r;
            }
            __syncthreads();
            // radial functions, one (order, point) per task; a point with k r >= 2 (large
            // leaves at high frequency) takes the whole recurrence in its order-0 task
            for (int task = threadIdx.x; task < (p + 1) * kChunk; task += blockDim.x) {
                const int n = task / kChunk, j = task % kChunk;
                if (j >= cnt) continue;
                const float x = rr[j];
                if (x < 2.0f) {
                    rad[j * (p + 1) + n] = f_jn_series(n, x, s);
                } else if (n == 0) {
                    float jr[HFMM_PMAX + 1];
                    f_jn_scaled(p, x, s, jr);
                    for (int q = 0; q <= p; ++q) rad[j * (p + 1) + q] = jr[q];
                }
            }
            __syncthreads();
            for (int task = threadIdx.x; task < (p + 1) * kChunk; task += blockDim.x) {
                const int mm = task / kChunk, j = task % kChunk;  // a warp shares one m
                if (j >= cnt) continue;
                const float ct = geo[4 * j], st = geo[4 * j + 1], ex = geo[4 * j + 2], ey = geo[4 * j + 3];
                float qmm = c_leg_qmm[mm], er = 1.f, ei = 0.f;
                for (int q = 0; q < mm; ++q) {
                    qmm *= st;
                    const float t = er * ex - ei * ey;
                    ei = er * ey + ei * ex;
                    er = t;
                }
                const float2 sg = sig[j0 + j];
                float* e = E + (j * (p + 1) + mm) * 4;
                e[0] = sg.x * er + sg.y * ei;  // sh e^{-i m phi}
                e[1] = sg.y * er - sg.x * ei;
                e[2] = sg.x * er - sg.y * ei;  // sh e^{+i m phi}
                e[3] = sg.y * er + sg.x * ei;
                const float* rj = rad + j * (p + 1);
                float* bj = B + j * H;
                float qa = qmm, qb = 0.f;
                bj[mm * (mm + 1) / 2 + mm] = rj[mm] * qmm;
                for (int nn = mm + 1; nn <= p; ++nn) {
                    const int h = nn * (nn + 1) / 2 + mm;
                    const float qn = (nn == mm + 1) ? c_leg_a[h] * ct * qmm : c_leg_a[h] * (ct * qa - c_leg_b[h] * qb);
                    qb = qa;
                    qa = qn;
                    bj[h] = rj[nn] * qn;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (cc[q] < P)
                    for (int t = 0; t < cnt; ++t) {
                        const float bb = B[t * H + hidx[q]];
                        const float* e = E + t * (p + 1) * 4;
                        accr[q] = fmaf(bb, e[eo[q]], accr[q]);
                        acci[q] = fmaf(bb, e[eo[q] + 1], acci[q]);
                    }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (cc[q] < P) M[box * P + cc[q]] = make_float2(accr[q], acci[q]);
    }
}

size_t p2m_smem_bytes(int p) {
    const int H = (p + 1) * (p + 2) / 2;
    return sizeof(float) * (32 * (p + 1) + 32 * H + 32 * (p + 1) * 4 + 128 + 32);
}

// ============================================================== L2P
__global__ void __launch_bounds__(128) k_l2p(int64_t N, const int32_t* __restrict__ pt_leaf,
                                             const float4* __restrict__ pts, int p, float s,
                                             const float2* __restrict__ Lc, float2* __restrict__ phi,
                                             const int32_t* __restrict__ leaf_lev, int lev,
                                             const int32_t* __restrict__ leaf_box) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t b = pt_leaf[i];
    if (leaf_lev && leaf_lev[b] != lev) return;  // adaptive tree: this launch's level only
    const int P = (p + 1) * (p + 1);
    const float2* L = Lc + (int64_t)(leaf_box ? leaf_box[b] : b) * P;
    const float4 y = pts[i];
    const Dir d = make_dir(y.x, y.y, y.z);
    float jr[HFMM_PMAX + 1];
    f_jn_scaled(p, d.r, s, jr);
    float accr = 0.f, acci = 0.f;
    float stp = 1.f, er = 1.f, ei = 0.f;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            stp *= d.st;
            const float t = er * d.ex - ei * d.ey;
            ei = er * d.ey + ei * d.ex;
            er = t;
        }
        const float qmm = c_leg_qmm[m] * stp;
        float qa = qmm, qb = 0.f;
        for (int n = m; n <= p; ++n) {
            float qn = qmm;
            if (n > m) {
                const int h = n * (n + 1) / 2 + m;
                qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                qb = qa;
                qa = qn;
            }
            const float bq = jr[n] * qn;
            const float2 lp = L[n * n + n + m];
            // L_{n,m} b e^{+i m phi}
            accr += bq * (lp.x * er - lp.y * ei);
            acci += bq * (lp.x * ei + lp.y * er);
            if (m > 0) {
                const float2 lm = L[n * n + n - m];
                accr += bq * (lm.x * er + lm.y * ei);
                acci += bq * (lm.y * er - lm.x * ei);
            }
        }
    }
    const float2 o = phi[i];
    phi[i] = make_float2(o.x + accr, o.y + acci);
}

// ============================================================== P2M / L2P at fixed order
// The leaf level's order is usually small (p <= 8, P <= 81): with p a template
// parameter every loop unrolls and the radial functions stay in registers.
constexpr int kFixedPMax = 8;

// jt_n(k r) / s^n, n = 0..PP, into registers
template <int PP>
__device__ __forceinline__ void jn_fixed(float x, float s, float (&jr)[PP + 1]) {
    if (x < 2.0f) {
#pragma unroll
        for (int n = 0; n <= PP; ++n) jr[n] = f_jn_series(n, x, s);
    } else {  // large leaves at high frequency: the downward recurrence
        float t[HFMM_PMAX + 1];
        f_jn_scaled(PP, x, s, t);
#pragma unroll
        for (int n = 0; n <= PP; ++n) jr[n] = t[n];
    }
}

// P2M, one warp per leaf (four leaves per block), the leaf's points in chunks of 32:
//   lane j builds the basis of point j: jt_n Q_n^m (m >= 0) into column j of Bs and
//   sh e^{-/+ i m phi} into column j of Es (row stride 33: lanes that read different
//   rows at one point hit different banks);
//   lane c then accumulates coefficients c, c + 32, ... over the chunk.
template <int PP>
__global__ void __launch_bounds__(128) k_p2m_w(int64_t nleaf, const int32_t* __restrict__ leaf_start,
                                               const float4* __restrict__ pts, const float2* __restrict__ sig,
                                               float s, float2* __restrict__ M, const int32_t* __restrict__ leaf_lev,
                                               int lev, const int32_t* __restrict__ leaf_box) {
    constexpr int P = (PP + 1) * (PP + 1), H = (PP + 1) * (PP + 2) / 2, NE = 2 * (PP + 1);
    constexpr int NC = (P + 31) / 32;
    __shared__ float Bs[4][H][33];
    __shared__ float2 Es[4][NE][33];
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t leaf = (int64_t)blockIdx.x * 4 + wb;
    if (leaf >= nleaf) return;  // warps are independent: no block-wide barrier below
    if (leaf_lev && leaf_lev[leaf] != lev) return;  // adaptive tree: this launch's level only
    const int64_t box = leaf_box ? leaf_box[leaf] : leaf;
    const int32_t b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    int hh[NC], ee[NC];
    float accr[NC], acci[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = min(lane + 32 * q, P - 1);
        int n = 0;
        while ((n + 1) * (n + 1) <= c) ++n;
        const int m = c - n * n - n, am = m < 0 ? -m : m;
        hh[q] = n * (n + 1) / 2 + am;
        ee[q] = m < 0 ? PP + 1 + am : am;
        accr[q] = acci[q] = 0.f;
    }
    for (int32_t j0 = b0; j0 < b1; j0 += 32) {
        const int cnt = min(32, b1 - j0);
        if (lane < cnt) {
            const float4 y = pts[j0 + lane];
            const float2 sg = sig[j0 + lane];
            const Dir d = make_dir(y.x, y.y, y.z);
            float jr[PP + 1];
            jn_fixed<PP>(d.r, s, jr);
            float stp = 1.f, er = 1.f, ei = 0.f;
#pragma unroll
            for (int m = 0; m <= PP; ++m) {
                if (m > 0) {
                    stp *= d.st;
                    const float t = er * d.ex - ei * d.ey;
                    ei = er * d.ey + ei * d.ex;
                    er = t;
                }
                const float qmm = c_leg_qmm[m] * stp;
                float qa = qmm, qb = 0.f;
                Bs[wb][m * (m + 1) / 2 + m][lane] = jr[m] * qmm;
#pragma unroll
                for (int n = m + 1; n <= PP; ++n) {
                    const int h = n * (n + 1) / 2 + m;
                    const float qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                    qb = qa;
                    qa = qn;
                    Bs[wb][h][lane] = jr[n] * qn;
                }
                Es[wb][m][lane] = make_float2(sg.x * er + sg.y * ei, sg.y * er - sg.x * ei);           // sh e^{-i m phi}
                Es[wb][PP + 1 + m][lane] = make_float2(sg.x * er - sg.y * ei, sg.y * er + sg.x * ei);  // sh e^{+i m phi}
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NC; ++q)
            for (int t = 0; t < cnt; ++t) {
                const float b = Bs[wb][hh[q]][t];
                const float2 e = Es[wb][ee[q]][t];
                accr[q] = fmaf(b, e.x, accr[q]);
                acci[q] = fmaf(b, e.y, acci[q]);
            }
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < NC; ++q)
        if (lane + 32 * q < P) M[box * P + lane + 32 * q] = make_float2(accr[q], acci[q]);
}

// L2P, one thread per point: phi += sum_nm L_nm jt_n(k r) Y_nm
template <int PP>
__global__ void __launch_bounds__(128) k_l2p_t(int64_t N, const int32_t* __restrict__ pt_leaf,
                                               const float4* __restrict__ pts, float s, const float2* __restrict__ Lc,
                                               float2* __restrict__ phi, const int32_t* __restrict__ leaf_lev, int lev,
                                               const int32_t* __restrict__ leaf_box) {
    constexpr int P = (PP + 1) * (PP + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t b = pt_leaf[i];
    if (leaf_lev && leaf_lev[b] != lev) return;  // adaptive tree: this launch's level only
    const float2* L = Lc + (int64_t)(leaf_box ? leaf_box[b] : b) * P;
    const float4 y = pts[i];
    const Dir d = make_dir(y.x, y.y, y.z);
    float jr[PP + 1];
    jn_fixed<PP>(d.r, s, jr);
    float accr = 0.f, acci = 0.f;
    float stp = 1.f, er = 1.f, ei = 0.f;
#pragma unroll
    for (int m = 0; m <= PP; ++m) {
        if (m > 0) {
            stp *= d.st;
            const float t = er * d.ex - ei * d.ey;
            ei = er * d.ey + ei * d.ex;
            er = t;
        }
        const float qmm = c_leg_qmm[m] * stp;
        float qa = qmm, qb = 0.f;
#pragma unroll
        for (int n = m; n <= PP; ++n) {
            float qn = qmm;
            if (n > m) {
                const int h = n * (n + 1) / 2 + m;
                qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                qb = qa;
                qa = qn;
            }
            const float bq = jr[n] * qn;
            const float2 lp = __ldg(L + n * n + n + m);
            // L_{n,m} b e^{+i m phi}
            accr += bq * (lp.x * er - lp.y * ei);
            acci += bq * (lp.x * ei + lp.y * er);
            if (m > 0) {
                const float2 lm = __ldg(L + n * n + n - m);
                accr += bq * (lm.x * er + lm.y * ei);
                acci += bq * (lm.y * er - lm.x * ei);
            }
        }
    }
    const float2 o = phi[i];
    phi[i] = make_float2(o.x + accr, o.y + acci);
}

// leaf filter of level l: every leaf of a uniform tree is at level L (no filter)
struct LeafFilter {
    const int32_t* lev;
    int l;
    const int32_t* box;
};
static LeafFilter leaf_filter(const hfmm_plan* P, int l) {
    return P->adaptive ? LeafFilter{P->leaf_lev.p, l, P->leaf_box.p} : LeafFilter{nullptr, l, nullptr};
}

template <int PP>
static void launch_p2m_l2p_fixed(bool p2m, const hfmm_plan* P, const LevelInfo& lv, LeafFilter f, cudaStream_t st) {
    if (p2m)
        k_p2m_w<PP><<<(unsigned)((P->nleaf + 3) / 4), 128, 0, st>>>(P->nleaf, P->leaf_start.p, P->pts.p, P->sig.p,
                                                                    (float)lv.s, P->coef.p + lv.mofs, f.lev, f.l, f.box);
    else
        k_l2p_t<PP><<<(unsigned)((P->N + 127) / 128), 128, 0, st>>>(P->N, P->pt_leaf.p, P->pts.p, (float)lv.s,
                                                                    P->coef.p + lv.lofs, P->phi.p, f.lev, f.l, f.box);
}

// P2M (p2m = true) or L2P of the leaves of one level at its fixed order; false if p > kFixedPMax
static bool p2m_l2p_fixed(bool p2m, const hfmm_plan* P, const LevelInfo& lv, LeafFilter f, cudaStream_t st) {
    switch (lv.p) {
        case 1: launch_p2m_l2p_fixed<1>(p2m, P, lv, f, st); return true;
        case 2: launch_p2m_l2p_fixed<2>(p2m, P, lv, f, st); return true;
        case 3: launch_p2m_l2p_fixed<3>(p2m, P, lv, f, st); return true;
        case 4: launch_p2m_l2p_fixed<4>(p2m, P, lv, f, st); return true;
        case 5: launch_p2m_l2p_fixed<5>(p2m, P, lv, f, st); return true;
        case 6: launch_p2m_l2p_fixed<6>(p2m, P, lv, f, st); return true;
        case 7: launch_p2m_l2p_fixed<7>(p2m, P, lv, f, st); return true;
        case 8: launch_p2m_l2p_fixed<8>(p2m, P, lv, f, st); return true;
        default: return false;
    }
}

// ============================================================== adaptive W lists (M2P, P2L)
// Singular functions of an expansion about a box centre, scaled like the translation
// operators: ht_n = h_n(x) s^(n+1), h_n = j_n + i y_n (n = 0..p).  y_n by its upward
// recurrence (stable), scaled: yt_{n+1} = (2n+1) s yt_n / x - s^2 yt_{n-1}.
__device__ void f_hn_scaled(int p, float x, float s, float* hr, float* hi) {
    float jr[HFMM_PMAX + 1];
    f_jn_scaled(p, x, s, jr);  // j_n / s^n
    float sn, cs;
    sincosf(x, &sn, &cs);
    const float s2 = s * s, inv = 1.0f / x;
    hi[0] = -cs * inv * s;
    if (p >= 1) hi[1] = (-cs * inv * inv - sn * inv) * s2;
    for (int n = 1; n < p; ++n) hi[n + 1] = (float)(2 * n + 1) * inv * s * hi[n] - s2 * hi[n - 1];
    float sp = s;
    for (int n = 0; n <= p; ++n) {
        hr[n] = jr[n] * sp;  // j_n s^(n+1)
        sp *= s2;
    }
}

// M2P: phi_i += (4 pi i / s_c) sum_nm M_nm(c) ht_n(k r) Y_nm(r^) over the W boxes c of the
// leaf of sorted point i, r = x_i - centre of c; M is the P2M kernels' multipole
// (sum_j sig_j jt_n conj Y_nm), so this is sum_j sig_j e^{ikR} / (kR) over c's points.
__global__ void __launch_bounds__(128) k_m2p(int64_t N, const int32_t* __restrict__ pt_leaf,
                                             const float4* __restrict__ pts, const int4* __restrict__ leaf_c2,
                                             const int32_t* __restrict__ w_ptr, const int4* __restrict__ w_c2,
                                             const int32_t* __restrict__ w_idx, const AdLevel* __restrict__ lev,
                                             float half_k, const float2* __restrict__ coef,
                                             float2* __restrict__ phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t b = pt_leaf[i];
    const int32_t q0 = w_ptr[b], q1 = w_ptr[b + 1];
    if (q0 == q1) return;
    const float4 y = pts[i];
    const int4 lc = leaf_c2[b];
    float hr[HFMM_PMAX + 1], hi[HFMM_PMAX + 1];
    float accr = 0.f, acci = 0.f;
    for (int32_t q = q0; q < q1; ++q) {
        const int4 c = w_c2[q];
        const AdLevel lv = lev[c.w];
        const int p = lv.p, P = (p + 1) * (p + 1);
        const float2* M = coef + lv.mofs + (int64_t)w_idx[q] * P;
        const Dir d = make_dir(y.x + (float)(lc.x - c.x) * half_k, y.y + (float)(lc.y - c.y) * half_k,
                               y.z + (float)(lc.z - c.z) * half_k);
        f_hn_scaled(p, d.r, lv.s, hr, hi);
        float sr = 0.f, si = 0.f;  // sum_nm M_nm ht_n Y_nm
        float stp = 1.f, er = 1.f, ei = 0.f;
        for (int m = 0; m <= p; ++m) {
            if (m > 0) {
                stp *= d.st;
                const float t = er * d.ex - ei * d.ey;
                ei = er * d.ey + ei * d.ex;
                er = t;
            }
            const float qmm = c_leg_qmm[m] * stp;
            float qa = qmm, qb = 0.f;
            for (int n = m; n <= p; ++n) {
                float qn = qmm;
                if (n > m) {
                    const int h = n * (n + 1) / 2 + m;
                    qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                    qb = qa;
                    qa = qn;
                }
                const float br = hr[n] * qn, bi = hi[n] * qn;
                const float2 mp = __ldg(M + n * n + n + m);  // M_{n,m} e^{+i m phi}
                const float a = mp.x * er - mp.y * ei, bb = mp.x * ei + mp.y * er;
                sr += br * a - bi * bb;
                si += br * bb + bi * a;
                if (m > 0) {  // M_{n,-m} e^{-i m phi}
                    const float2 mm = __ldg(M + n * n + n - m);
                    const float a2 = mm.x * er + mm.y * ei, b2 = mm.y * er - mm.x * ei;
                    sr += br * a2 - bi * b2;
                    si += br * b2 + bi * a2;
                }
            }
        }
        const float f = 12.566370614359172f / lv.s;  // 4 pi / s, times i below
        accr -= f * si;
        acci += f * sr;
    }
    const float2 o = phi[i];
    phi[i] = make_float2(o.x + accr, o.y + acci);
}

// P2L: L_nm(c) += (4 pi i / s_c) sum_j sig_j ht_n(k r_j) conj Y_nm(r_j^) for the points j of
// the leaf that owns W entry e (block e), r_j = y_j - centre of c.  The leaf's points are
// taken in chunks: thread j writes its point's row sig_j ht_n Q_n^|m| e^{-/+ i m phi} (P
// values, row stride P + 1) into shared memory, then thread q sums coefficient q over the
// chunk; one reduction per coefficient reaches the locals.
constexpr int kP2LMaxPerThread = 8;  // coefficients per thread: P <= 8 * 128 (orders <= 30)
__global__ void __launch_bounds__(128) k_p2l(const int32_t* __restrict__ w_leaf, const int4* __restrict__ w_c2,
                                             const int32_t* __restrict__ w_idx, const AdLevel* __restrict__ lev,
                                             const int32_t* __restrict__ leaf_start,
                                             const int4* __restrict__ leaf_c2, const float4* __restrict__ pts,
                                             const float2* __restrict__ sig, float half_k, int chunk,
                                             float2* __restrict__ coef) {
    extern __shared__ float2 rows_p2l[];  // [chunk][P + 1]
    const int e = blockIdx.x;
    const int32_t t = w_leaf[e];
    const int4 c = w_c2[e];
    const AdLevel lv = lev[c.w];
    const int p = lv.p, P = (p + 1) * (p + 1), stride = P + 1;
    const int4 lc = leaf_c2[t];
    const int32_t j0 = leaf_start[t], j1 = leaf_start[t + 1];
    float2 acc[kP2LMaxPerThread];
#pragma unroll
    for (int u = 0; u < kP2LMaxPerThread; ++u) acc[u] = make_float2(0.f, 0.f);
    float hr[HFMM_PMAX + 1], hi[HFMM_PMAX + 1];
    for (int32_t jb = j0; jb < j1; jb += chunk) {
        const int cnt = min(chunk, j1 - jb);
        __syncthreads();  // the previous chunk's rows are summed
        for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) {
            const float4 y = pts[jb + jj];
            const float2 g = sig[jb + jj];
            float2* row = rows_p2l + jj * stride;
            const Dir d = make_dir(y.x + (float)(lc.x - c.x) * half_k, y.y + (float)(lc.y - c.y) * half_k,
                                   y.z + (float)(lc.z - c.z) * half_k);
            f_hn_scaled(p, d.r, lv.s, hr, hi);
            float stp = 1.f, er = 1.f, ei = 0.f;
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    stp *= d.st;
                    const float tt = er * d.ex - ei * d.ey;
                    ei = er * d.ey + ei * d.ex;
                    er = tt;
                }
                const float qmm = c_leg_qmm[m] * stp;
                float qa = qmm, qb = 0.f;
                for (int n = m; n <= p; ++n) {
                    float qn = qmm;
                    if (n > m) {
                        const int h = n * (n + 1) / 2 + m;
                        qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                        qb = qa;
                        qa = qn;
                    }
                    const float br = hr[n] * qn, bi = hi[n] * qn;
                    const float u = g.x * br - g.y * bi, v = g.x * bi + g.y * br;  // sig ht_n Q
                    row[n * n + n + m] = make_float2(u * er + v * ei, v * er - u * ei);  // e^{-i m phi}
                    if (m > 0) row[n * n + n - m] = make_float2(u * er - v * ei, v * er + u * ei);  // e^{+i m phi}
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kP2LMaxPerThread; ++u) {
            const int q = threadIdx.x + u * blockDim.x;
            if (q < P)
                for (int jj = 0; jj < cnt; ++jj) {
                    const float2 r = rows_p2l[jj * stride + q];
                    acc[u].x += r.x;
                    acc[u].y += r.y;
                }
        }
    }
    const float f = 12.566370614359172f / lv.s;
    float2* L = coef + lv.lofs + (int64_t)w_idx[e] * P;
#pragma unroll
    for (int u = 0; u < kP2LMaxPerThread; ++u) {  // times 4 pi i / s
        const int q = threadIdx.x + u * blockDim.x;
        if (q < P) red_add(L + q, make_float2(-f * acc[u].y, f * acc[u].x));
    }
}

// rows of the chunk that fit 24 KiB of shared memory
static int p2l_chunk(int P) { return std::max(1, std::min(32, 24576 / (8 * (P + 1)))); }

// ============================================================== batched translations
// Out[:, dst] += T * In[:, src] for the column pairs of one work item.
// 128 threads; a block computes one output tile of 4 * (128 / CG) rows x 4 * CG
// columns (blockIdx.y selects the rows), each thread 4 rows x 4 columns, with K
// in slices staged in shared memory.  CG = 16 (32 x 64 tiles) serves items with
// many columns; CG = 4 (128 x 16) and CG = 2 (256 x 8) serve the coarse levels,
// where an offset has only a few targets and the high order makes T the large
// operand.  Row tiles in separate blocks let a level with few items fill the GPU.
// rhs > 1: batched items (one box pair standing for the columns box * rhs + c).
// Four blocks per SM (at most 128 registers, no spills): 0.192 -> 0.179 ms for the SIMT M2L
// of the 1.97 M-point workload against the unconstrained 134-168 registers (three blocks).
template <int CG>
__global__ void __launch_bounds__(128, 4) k_translate(const TransItem* __restrict__ items, int64_t item0,
                                                   const int2* __restrict__ cols, const float2* __restrict__ ops,
                                                   float2* __restrict__ coef, int rhs) {
    constexpr int RG = 128 / CG;             // row groups
    constexpr int TR = 4 * RG, TC = 4 * CG;  // tile rows, tile columns
    constexpr int KS = TR >= 128 ? 2048 / TR : 32;  // K slice: <= 16 T elements per thread
    __shared__ float2 sT[TR][KS + 1];
    __shared__ float2 sX[KS][TC + 1];
    __shared__ int2 sc[TC];
    TransItem it = items[item0 + blockIdx.x];
    int tid = threadIdx.x;
    int ncol = it.ncol, Pin = it.pin, Pout = it.pout;
    const int r0 = TR * (int)blockIdx.y;
    if (r0 >= Pout) return;  // uniform over the block: items of a lower order in the same launch
    // blockIdx.z: a range of K (launched only for accumulating items, whose outputs are reductions)
    const int kchunk = ((Pin + (int)gridDim.z - 1) / (int)gridDim.z + KS - 1) / KS * KS;
    const int kb = kchunk * (int)blockIdx.z, ke = min(Pin, kb + kchunk);
    if (kb >= ke) return;
    if (tid < TC) {
        int2 v = make_int2(0, 0);
        if (tid < ncol) {
            if (rhs > 1) {
                const int2 pr = cols[it.cols];
                v = make_int2(pr.x * rhs + tid, pr.y * rhs + tid);
            } else {
                v = cols[it.cols + tid];
            }
        }
        sc[tid] = v;
    }
    __syncthreads();
    const float2* T = ops + it.op;
    const int tx = tid % CG, ty = tid / CG;
    float accr[4][4], acci[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accr[a][b] = acci[a][b] = 0.f;
    // A slice's tiles pass through registers: every load of the next slice is issued
    // before the current slice is multiplied, so the loads overlap the arithmetic.
    constexpr int NT = TR * KS / 128, NX = (KS * TC + 127) / 128;
    float2 rT[NT], rX[NX];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int e = tid + 128 * q, rr = e / KS, kk = e % KS;
            const int r = r0 + rr, kq = k0 + kk;
            rT[q] = (r < Pout && kq < ke) ? __ldg(T + (int64_t)r * Pin + kq) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NX; ++q) {
            const int e = tid + 128 * q, cc = e / KS, kk = e % KS;
            const int kq = k0 + kk;
            rX[q] = (e < KS * TC && cc < ncol && kq < ke) ? __ldg(coef + it.src + (int64_t)sc[cc].x * Pin + kq)
                                                          : make_float2(0.f, 0.f);
        }
    };
    fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += KS) {
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int e = tid + 128 * q;
            sT[e / KS][e % KS] = rT[q];
        }
#pragma unroll
        for (int q = 0; q < NX; ++q) {
            const int e = tid + 128 * q;
            if (e < KS * TC) sX[e % KS][e / KS] = rX[q];
        }
        __syncthreads();
        if (k0 + KS < ke) fetch(k0 + KS);
#pragma unroll 8
        for (int kk = 0; kk < KS; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = sT[ty + RG * q][kk];
                b[q] = sX[kk][tx + CG * q];
            }
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) {
                    accr[qa][qb] = fmaf(a[qa].x, b[qb].x, fmaf(-a[qa].y, b[qb].y, accr[qa][qb]));
                    acci[qa][qb] = fmaf(a[qa].x, b[qb].y, fmaf(a[qa].y, b[qb].x, acci[qa][qb]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
        int r = r0 + ty + RG * qa;
        if (r >= Pout) continue;
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            int cc = tx + CG * qb;
            if (cc >= ncol) continue;
            float2* o = coef + it.dst + (int64_t)sc[cc].y * Pout + r;
            if (it.atomic) {
                red_add(o, make_float2(accr[qa][qb], acci[qa][qb]));
            } else {
                float2 v = *o;
                *o = make_float2(v.x + accr[qa][qb], v.y + acci[qa][qb]);
            }
        }
    }
}

// ============================================================== correction (CSR SpMV)
// kCorrLanes lanes per row (rows hold ~3 * (near triangles) nonzeros, a few dozen), each
// taking kCorrUnroll nonzeros per pass.  Measured on the 1.97 M-point workload: 4 lanes x 8
// nonzeros 0.186 ms, 4 x 4 0.193 ms, 8 x 4 0.215 ms, 2 x 8 0.215 ms, 16 x 4 0.346 ms.
constexpr int kCorrLanes = 4;
constexpr int kCorrUnroll = 8;
__global__ void __launch_bounds__(256) k_corr(int64_t N, const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col, const float2* __restrict__ val,
                                              const float2* __restrict__ sig, float2* __restrict__ phi) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / kCorrLanes;
    const int sub = (int)(t % kCorrLanes);
    const bool active = row < N;
    float ar = 0.f, ai = 0.f;
    if (active) {
        const int64_t e0 = __ldg(ptr + row), e1 = __ldg(ptr + row + 1);
        int64_t e = e0 + sub;
        // kCorrUnroll nonzeros per lane per pass: their loads are all in flight together
        for (; e + (kCorrUnroll - 1) * kCorrLanes < e1; e += kCorrUnroll * kCorrLanes) {
            int32_t c[kCorrUnroll];
            float2 v[kCorrUnroll], g[kCorrUnroll];
#pragma unroll
            for (int q = 0; q < kCorrUnroll; ++q) {
                c[q] = __ldg(col + e + q * kCorrLanes);
                v[q] = __ldg(val + e + q * kCorrLanes);
            }
#pragma unroll
            for (int q = 0; q < kCorrUnroll; ++q) g[q] = __ldg(sig + c[q]);
#pragma unroll
            for (int q = 0; q < kCorrUnroll; ++q) {
                ar = fmaf(v[q].x, g[q].x, fmaf(-v[q].y, g[q].y, ar));
                ai = fmaf(v[q].x, g[q].y, fmaf(v[q].y, g[q].x, ai));
            }
        }
        for (; e < e1; e += kCorrLanes) {
            const float2 v = __ldg(val + e);
            const float2 g = __ldg(sig + __ldg(col + e));
            ar = fmaf(v.x, g.x, fmaf(-v.y, g.y, ar));
            ai = fmaf(v.x, g.y, fmaf(v.y, g.x, ai));
        }
    }
#pragma unroll
    for (int o = kCorrLanes / 2; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (active && sub == 0) {
        const float2 v = phi[row];
        phi[row] = make_float2(v.x + ar, v.y + ai);
    }
}

static void launch_corr(hfmm_plan* P, cudaStream_t st) {
    const int64_t threads = P->N * kCorrLanes;
    k_corr<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P->N, P->corr_ptr.p, P->corr_col.p, P->corr_val.p,
                                                              P->sig.p, P->phi.p);
    ++P->launches;
}

// ============================================================== direct O(N^2) sum
// Every target against every source (sorted order), leaf-local coordinates so
// close pairs keep their precision.
__global__ void __launch_bounds__(256) k_direct(int64_t N, const float4* __restrict__ pts,
                                                const int32_t* __restrict__ pt_leaf,
                                                const int4* __restrict__ leaf_ijk, const float2* __restrict__ sig,
                                                float shift, float2* __restrict__ phi) {
    __shared__ float4 sp[256];
    __shared__ float2 sg[256];
    __shared__ int4 sl[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < N;
    float4 t = active ? pts[i] : make_float4(0, 0, 0, 0);
    int4 tij = active ? leaf_ijk[pt_leaf[i]] : make_int4(0, 0, 0, 0);
    float ar = 0.f, ai = 0.f;
    for (int64_t j0 = 0; j0 < N; j0 += 256) {
        int64_t j = j0 + threadIdx.x;
        if (j < N) {
            sp[threadIdx.x] = pts[j];
            sg[threadIdx.x] = sig[j];
            sl[threadIdx.x] = leaf_ijk[pt_leaf[j]];
        }
        __syncthreads();
        int cnt = (N - j0 < 256) ? (int)(N - j0) : 256;
        for (int q = 0; q < cnt; ++q) {
            if (j0 + q == i) continue;
            float4 s = sp[q];
            int4 l = sl[q];
            float dx = fmaf((float)(tij.x - l.x), shift, t.x) - s.x;
            float dy = fmaf((float)(tij.y - l.y), shift, t.y) - s.y;
            float dz = fmaf((float)(tij.z - l.z), shift, t.z) - s.z;
            float u = dx * dx + dy * dy + dz * dz;
            if (u == 0.f) continue;
            float rinv = rsqrtf(u), r = u * rinv, sn, cs;
            sincosf(r, &sn, &cs);
            float re = cs * rinv, im = sn * rinv;
            float2 g = sg[q];
            ar += g.x * re - g.y * im;
            ai += g.x * im + g.y * re;
        }
        __syncthreads();
    }
    if (active) phi[i] = make_float2(ar, ai);
}

__global__ void k_planewave(int64_t N, const double* __restrict__ x64, double k, double dx, double dy, double dz,
                            float2* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double ph = k * (dx * x64[3 * i] + dy * x64[3 * i + 1] + dz * x64[3 * i + 2]);
    double s, c;
    sincos(ph, &s, &c);
    out[i] = make_float2((float)c, (float)s);
}

void launch_planewave(hfmm_plan* P, double dx, double dy, double dz, float2* out, cudaStream_t st) {
    ++P->launches;
    k_planewave<<<(unsigned)((P->N + 255) / 256), 256, 0, st>>>(P->N, P->x64.p, P->k, dx, dy, dz, out);
}

// ============================================================== drivers
void mark_stage(hfmm_plan* P, int q, cudaStream_t st) {
    if (P->stage_ev) HFMM_CUDA(cudaEventRecord(P->stage_ev[q], st));
}

// Items [b, e) of at most `width` columns (64, 16 or 8) and output order <= pout_max; kparts > 1
// splits K across blocks and needs accumulating (atomic) items.
static void launch_translate(hfmm_plan* P, const TransItem* items, float2* coef, int rhs, int64_t b, int64_t e,
                             int pout_max, int width, cudaStream_t st, int kparts = 1) {
    if (e <= b) return;
    const int rows = width > 16 ? 32 : width > 8 ? 128 : 256;
    const dim3 grid((unsigned)(e - b), (unsigned)((pout_max + rows - 1) / rows), (unsigned)kparts);
    if (width > 16)
        k_translate<16><<<grid, 128, 0, st>>>(items, b, P->item_cols.p, P->ops.p, coef, rhs);
    else if (width > 8)
        k_translate<4><<<grid, 128, 0, st>>>(items, b, P->item_cols.p, P->ops.p, coef, rhs);
    else
        k_translate<2><<<grid, 128, 0, st>>>(items, b, P->item_cols.p, P->ops.p, coef, rhs);
    ++P->launches;
}

static int p2p_sm_count();

// M2M / L2L between the coarse levels: few items (8 offsets) of many rows, so K is split
// across blocks until about two blocks per SM are in flight, each part at least 32 deep
// (the items accumulate, so the parts' partial sums add in the output).
static void launch_tree_translate(hfmm_plan* P, const TransItem* items, float2* coef, int rhs, int64_t b, int64_t e,
                                  int pout, int pin, cudaStream_t st) {
    const int64_t blocks = (e - b) * ((pout + 31) / 32);
    int kparts = 1;
    if (blocks > 0) {
        const int64_t want = (2 * (int64_t)p2p_sm_count() + blocks - 1) / blocks;
        kparts = (int)std::max<int64_t>(1, std::min<int64_t>(want, pin / 32));
    }
    launch_translate(P, items, coef, rhs, b, e, pout, HFMM_TRANS_NB, st, kparts);
}

// Near field (P2P between neighbouring leaves, or zeros): the first writer of P->phi.
static int p2p_sm_count() {
    static int n[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 0;
    if (!n[dev]) HFMM_CUDA(cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev));
    return n[dev];
}

static void near_stage(hfmm_plan* P, int parts, cudaStream_t st) {
    int64_t N = P->N;
    mark_stage(P, 1, st);
    if (parts & 1) {
        const size_t staged = (size_t)P->p2p_cap * (sizeof(float4) + sizeof(float));
        if (P->p2p_cap > 0 && staged <= 96 * 1024 && P->p2p_maxnbr <= kStagedNbr) {
            const int cap_pairs = P->p2p_cap / 2 + 2;
            const size_t pk_smem = (size_t)cap_pairs * (2 * sizeof(float4) + sizeof(float2));
            if (P->poly_p2p && P->p2p_variant == 2) {
                const int grid = (int)std::min<int64_t>(P->nleaf, (int64_t)kPipeBlocksPerSM * p2p_sm_count());
                k_p2p_pipe<<<(unsigned)grid, kPkThreads, (size_t)cap_pairs * (4 * sizeof(float4) + 3 * sizeof(float2)),
                             st>>>((int)P->nleaf, P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p, P->pts.p,
                                   P->sig.p, P->p2p_shift, cap_pairs, P->phi.p);
            } else if (P->poly_p2p && P->p2p_variant == 1) {
                k_p2p_packed<kPkTargets><<<(unsigned)P->nleaf, kPkThreads, pk_smem, st>>>(
                    P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift,
                    cap_pairs, P->phi.p);
            } else if (P->poly_p2p)
                k_p2p_staged<true><<<(unsigned)P->nleaf, 128, staged, st>>>(
                    P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift,
                    P->p2p_cap, P->phi.p);
            else
                k_p2p_staged<false><<<(unsigned)P->nleaf, 128, staged, st>>>(
                    P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift,
                    P->p2p_cap, P->phi.p);
        } else {
        unsigned nb = (unsigned)((P->ntiles * 32 + 255) / 256);
        if (P->poly_p2p)
            k_p2p<true><<<nb, 256, 0, st>>>(P->ntiles, P->tiles.p, P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p,
                                            P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift, P->phi.p);
        else
            k_p2p<false><<<nb, 256, 0, st>>>(P->ntiles, P->tiles.p, P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p,
                                             P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift, P->phi.p);
        }
        ++P->launches;
    } else {
        HFMM_CUDA(cudaMemsetAsync(P->phi.p, 0, sizeof(float2) * N, st));
    }
}

// Far field up to the leaves' locals: P2M (and P2L), M2M (and M2P), M2L, L2L.
static void far_stage(hfmm_plan* P, int parts, cudaStream_t st) {
    int64_t N = P->N;
    mark_stage(P, 2, st);
    int L = P->L;
    bool far = (parts & 2) && L >= 2;
    if (far) {
        // multipoles above the leaves and all locals accumulate: clear them
        HFMM_CUDA(cudaMemsetAsync(P->coef.p, 0, sizeof(float2) * P->coef_total, st));
        for (int l : P->leaf_levels) {  // the leaves of each level (all at L in a uniform tree)
            const LevelInfo& lv = P->lev[l];
            const LeafFilter f = leaf_filter(P, l);
            if (!p2m_l2p_fixed(true, P, lv, f, st)) {
                const size_t smem = p2m_smem_bytes(lv.p);
                k_p2m<<<(unsigned)P->nleaf, 128, smem, st>>>(P->leaf_start.p, P->pts.p, P->sig.p, lv.p, (float)lv.s,
                                                               P->coef.p + lv.mofs, f.lev, f.l, f.box);
            }
            ++P->launches;
        }
        if (P->adaptive && P->n_w > 0) {  // W lists: the leaf's points into the W boxes' locals
            const int chunk = p2l_chunk(P->w_maxP);
            k_p2l<<<(unsigned)P->n_w, 128, sizeof(float2) * chunk * (P->w_maxP + 1), st>>>(
                P->w_leaf.p, P->w_c2.p, P->w_idx.p, P->ad_lev.p, P->leaf_start.p, P->leaf_ijk.p, P->pts.p, P->sig.p,
                P->p2p_shift, chunk, P->coef.p);
            ++P->launches;
        }
    }
    mark_stage(P, 3, st);
    if (far)
        for (int l = L - 1; l >= 2; --l) {
            const auto& g = P->m2m_tc[l];
            if (g.second > g.first) {
                m2l_tc_launch(P->tc_groups.p + g.first, g.second - g.first, P->items.p, P->item_cols.p, P->aops.p,
                              P->coef.p, P->dev_err.p, 1, st);
                ++P->launches;
            } else {
                launch_tree_translate(P, P->items.p, P->coef.p, 1, P->m2m_items_begin[l], P->m2m_items_end[l],
                                      P->lev[l].P, P->lev[l + 1].P, st);
            }
        }
    if (far && P->adaptive && P->n_w > 0) {  // W lists: the W boxes' multipoles at the leaf's points
        k_m2p<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(N, P->pt_leaf.p, P->pts.p, P->leaf_ijk.p, P->w_ptr.p,
                                                           P->w_c2.p, P->w_idx.p, P->ad_lev.p, P->p2p_shift,
                                                           P->coef.p, P->phi.p);
        ++P->launches;
    }
    mark_stage(P, 4, st);
    if (far)
        for (const SimtRange& r : P->m2l_simt)  // high orders: K in 2-3 parts for more blocks in flight
            launch_translate(P, P->items.p, P->coef.p, 1, r.begin, r.end, r.pout_max, r.width, st,
                             r.pout_max >= 200 ? 3 : r.pout_max >= 100 ? 2 : 1);
    mark_stage(P, 5, st);
    if (far) {
        if (P->m2l_variant == 1 && P->n_ts_tiles > 0) {
            m2l_ts_split(P->ts_split, P->ts_split_boxes, P->coef.p, P->ts_bx.p, st);
            m2l_ts_launch(P->ts_tiles.p, P->n_ts_tiles, P->ts_max_chunks, P->ts_chunks.p, P->ts_cols.p,
                          P->m2l_canon.p, P->ts_bx.p, P->coef.p, P->dev_err.p, st);
            P->launches += 2;
        } else if (P->n_tc_groups > 0) {
            m2l_tc_launch(P->tc_groups.p, P->n_tc_groups, P->items.p, P->item_cols.p, P->aops.p, P->coef.p,
                          P->dev_err.p, 1, st);
            ++P->launches;
        }
    }
    mark_stage(P, 6, st);
    if (far)
        for (int l = 3; l <= L; ++l) {
            const auto& g = P->l2l_tc[l];
            if (g.second > g.first) {
                m2l_tc_launch(P->tc_groups.p + g.first, g.second - g.first, P->items.p, P->item_cols.p, P->aops.p,
                              P->coef.p, P->dev_err.p, 1, st);
                ++P->launches;
            } else {
                launch_tree_translate(P, P->items.p, P->coef.p, 1, P->l2l_items_begin[l], P->l2l_items_end[l],
                                      P->lev[l].P, P->lev[l - 1].P, st);
            }
        }
}

// L2P: the leaves' locals at their points, added into P->phi.
static void l2p_stage(hfmm_plan* P, int parts, cudaStream_t st) {
    int64_t N = P->N;
    const int L = P->L;
    const bool far = (parts & 2) && L >= 2;
    mark_stage(P, 7, st);
    if (far) {
        for (int l : P->leaf_levels) {
            const LevelInfo& lv = P->lev[l];
            const LeafFilter f = leaf_filter(P, l);
            if (!p2m_l2p_fixed(false, P, lv, f, st))
                k_l2p<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(N, P->pt_leaf.p, P->pts.p, lv.p, (float)lv.s,
                                                                   P->coef.p + lv.lofs, P->phi.p, f.lev, f.l, f.box);
            ++P->launches;
        }
    }
}

// Near/self correction added into P->phi.
static void corr_stage(hfmm_plan* P, int parts, cudaStream_t st) {
    mark_stage(P, 8, st);
    if ((parts & 4) && P->corr_nnz > 0) {
        launch_corr(P, st);
    }
    mark_stage(P, 9, st);
    HFMM_CUDA(cudaGetLastError());
}


// Once per device, before any capture: the near-field and P2M kernels may take up to the
// device's opt-in shared memory per block (the launch decides how much it actually uses).
void matvec_kernels_init() {
    static bool done[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return;
    int optin = 0;
    HFMM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // the dynamic limit is what the opt-in maximum leaves beside the kernel's static shared memory
    auto allow = [&](const void* fn) {
        cudaFuncAttributes fa{};
        HFMM_CUDA(cudaFuncGetAttributes(&fa, fn));
        HFMM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       optin - (int)fa.sharedSizeBytes));
    };
    allow((const void*)k_p2p_staged<true>);
    allow((const void*)k_p2p_staged<false>);
    allow((const void*)k_p2p_packed<kPkTargets>);
    allow((const void*)k_p2p_pipe);
    allow((const void*)k_p2m);
    if (dev >= 0 && dev < 64) done[dev] = true;
}

// The four stages in order: every partial matvec and the stage-timed one run this way.
static void matvec_sequential(hfmm_plan* P, int parts, cudaStream_t st) {
    near_stage(P, parts, st);
    far_stage(P, parts, st);
    l2p_stage(P, parts, st);
    corr_stage(P, parts, st);
}

// Two branches: the near field and the correction (both only touch sig and phi) on a side
// stream beside the far field (sig -> coef); L2P, the last writer of phi, joins them.
static void matvec_branches(hfmm_plan* P, cudaStream_t st, cudaStream_t side) {
    MatvecGraph& G = P->mvg;
    HFMM_CUDA(cudaEventRecord(G.fork, st));
    HFMM_CUDA(cudaStreamWaitEvent(side, G.fork, 0));
    near_stage(P, 7, side);
    corr_stage(P, 7, side);
    HFMM_CUDA(cudaEventRecord(G.join, side));
    far_stage(P, 7, st);
    HFMM_CUDA(cudaStreamWaitEvent(st, G.join, 0));
    l2p_stage(P, 7, st);
}

// Captures fn's launches on `cap` (thread-local mode) into an instantiated graph.  Another
// thread of the process can invalidate a capture in progress (a device-wide synchronisation,
// as a memory release performs, while this thread is capturing); the capture is then
// abandoned, the error cleared, and false returned so the caller runs the work directly.
// Errors that are not about the capture propagate as usual.
template <typename Fn>
static bool capture_graph(cudaStream_t cap, Fn fn, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    HFMM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    bool ok = true;
    try {
        fn();
    } catch (const HfmmError&) {
        ok = false;
    }
    const cudaError_t ee = cudaStreamEndCapture(cap, &g);
    if (!ok || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        const cudaError_t last = cudaGetLastError();  // clears a non-sticky capture error
        const bool capture_err = ee == cudaErrorStreamCaptureInvalidated || last == cudaErrorStreamCaptureInvalidated ||
                                 ee == cudaErrorStreamCaptureUnsupported || last == cudaErrorStreamCaptureUnsupported;
        if (!capture_err && last != cudaSuccess) HFMM_CUDA(last);
        if (!capture_err && ee != cudaSuccess) HFMM_CUDA(ee);
        return false;
    }
    const cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    HFMM_CUDA(e);
    return true;
}

// sig (sorted, pre-scaled densities) -> phi (sorted potentials) for the whole operator.
// On uniform trees the matvec (the two-branch form for mv_mode 1, the chain of stages for
// mv_mode 0) is captured once per plan into a CUDA graph on a plan-owned stream and replayed
// on `st`: it reads and writes only plan-owned buffers, so one capture serves every later
// matvec, including the solver's.
void run_matvec_sorted(hfmm_plan* P, int parts, cudaStream_t st) {
    if (parts != 7 || P->stage_ev || P->adaptive) {
        matvec_sequential(P, parts, st);
        return;
    }
    // the whole matvec as one graph launch (two branches, or one chain): GMRES waits on the host
    // once per iteration, after which a chain of separate launches would leave the device idle
    // between the short tree-pass kernels while the host catches up
    MatvecGraph& G = P->mvg;
    const bool br = P->mv_mode == 1;
    cudaGraphExec_t& gx = br ? G.graph : G.seq;
    int64_t& gl = br ? G.launches : G.seq_launches;
    if (!gx) {
        if (!G.cap) HFMM_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
        if (!G.side) HFMM_CUDA(cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking));
        if (!G.fork) HFMM_CUDA(cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming));
        if (!G.join) HFMM_CUDA(cudaEventCreateWithFlags(&G.join, cudaEventDisableTiming));
        const int64_t l0 = P->launches;
        const bool ok = br ? capture_graph(G.cap, [&] { matvec_branches(P, G.cap, G.side); }, &gx)
                           : capture_graph(G.cap, [&] { matvec_sequential(P, 7, G.cap); }, &gx);
        if (!ok) {
            P->launches = l0;  // the capture was invalidated (see capture_graph): run the stages directly
            matvec_sequential(P, parts, st);
            return;
        }
        gl = P->launches - l0;
        P->launches = l0;
    }
    HFMM_CUDA(cudaGraphLaunch(gx, st));
    P->launches += gl;
}

void run_direct_sorted(hfmm_plan* P, cudaStream_t st) {
    int64_t N = P->N;
    k_direct<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, P->pts.p, P->pt_leaf.p, P->leaf_ijk.p, P->sig.p,
                                                          P->p2p_shift, P->phi.p);
    ++P->launches;
    if (P->corr_nnz > 0) {
        launch_corr(P, st);
    }
    HFMM_CUDA(cudaGetLastError());
}

// ============================================================== batched right-hand sides
// R = 2..64 right-hand sides in one matvec.  Densities and potentials are held
// [point][rhs] and expansions [box][rhs][P]: the R values a kernel needs for one
// point or one box are one contiguous block.  The near field evaluates each
// Green's-function tile once and multiplies it into all R densities; P2M and
// L2P become small complex GEMMs over R; the translations reuse the single
// right-hand-side kernels with one work item per box pair and R columns.
constexpr int kBMax = 64;    // right-hand sides per batched matvec
constexpr int kBChunk = 32;  // sources (P2P) or points (P2M, L2P) per shared-memory chunk
constexpr int kBMaxP = 128;  // leaf expansion size the batched P2M / L2P kernels take

// Regular basis b_c(y) = jt_n(r) Q_n^|m|(cos t) e^{i m phi}, c = n^2 + n + m, of a point y
// relative to its leaf centre (scaled by k):  L2P is sum_c L_c b_c,  P2M is sum_j s_j conj(b_c(y_j)).
// PP >= 0: the order as a compile-time constant (p is then PP), loops unrolled and the
// radial functions in registers; PP < 0: any order p
template <int PP>
__device__ void regular_basis(float4 y, int p, float s, float2* out) {
    const Dir d = make_dir(y.x, y.y, y.z);
    constexpr int kJ = PP >= 0 ? PP + 1 : HFMM_PMAX + 1;
    float jr[kJ];
    if constexpr (PP >= 0) {
        p = PP;
        jn_fixed<PP>(d.r, s, jr);
    } else {
        f_jn_scaled(p, d.r, s, jr);
    }
    float stp = 1.f, er = 1.f, ei = 0.f;
#pragma unroll
    for (int m = 0; m <= (PP >= 0 ? PP : p); ++m) {
        if (m > 0) {
            stp *= d.st;
            const float t = er * d.ex - ei * d.ey;
            ei = er * d.ey + ei * d.ex;
            er = t;
        }
        const float qmm = c_leg_qmm[m] * stp;
        float qa = qmm, qb = 0.f;
#pragma unroll
        for (int n = m; n <= (PP >= 0 ? PP : p); ++n) {
            float qn = qmm;
            if (n > m) {
                const int h = n * (n + 1) / 2 + m;
                qn = (n == m + 1) ? c_leg_a[h] * d.ct * qmm : c_leg_a[h] * (d.ct * qa - c_leg_b[h] * qb);
                qb = qa;
                qa = qn;
            }
            const float bq = jr[n] * qn;
            out[n * n + n + m] = make_float2(bq * er, bq * ei);
            if (m > 0) out[n * n + n - m] = make_float2(bq * er, -bq * ei);
        }
    }
}

// sig_b[i][r] = k w_i / (4 pi) density[r][perm_i]; 32 points per block, transposed in shared memory
__global__ void __launch_bounds__(256) k_prep_b(int64_t N, int R, const int32_t* __restrict__ perm,
                                                const float* __restrict__ wscale, const float2* __restrict__ dens,
                                                float2* __restrict__ sig) {
    __shared__ float2 t[32][kBMax + 1];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int ii = threadIdx.x & 31;
    const int64_t i = i0 + ii;
    const int32_t pi = i < N ? perm[i] : 0;
    for (int r = threadIdx.x >> 5; r < R; r += 8) t[ii][r] = i < N ? dens[(int64_t)r * N + pi] : make_float2(0.f, 0.f);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * R; e += 256) {
        const int a = e / R, r = e % R;
        const int64_t row = i0 + a;
        if (row < N) {
            const float w = wscale[row];
            const float2 v = t[a][r];
            sig[row * R + r] = make_float2(w * v.x, w * v.y);
        }
    }
}

// out[r][perm_i] = phi_b[i][r]
__global__ void __launch_bounds__(256) k_output_b(int64_t N, int R, const int32_t* __restrict__ perm,
                                                  const float2* __restrict__ phi, float2* __restrict__ out) {
    __shared__ float2 t[32][kBMax + 1];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    for (int e = threadIdx.x; e < 32 * R; e += 256) {
        const int a = e / R, r = e % R;
        const int64_t row = i0 + a;
        t[a][r] = row < N ? phi[row * R + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int ii = threadIdx.x & 31;
    const int64_t i = i0 + ii;
    if (i >= N) return;
    const int32_t pi = perm[i];
    for (int r = threadIdx.x >> 5; r < R; r += 8) out[(int64_t)r * N + pi] = t[ii][r];
}

// Near field for R right-hand sides: one block (8 warps) per target leaf.  Neighbour
// sources are staged (positions in the leaf's frame, global index); per chunk of 32
// sources the block evaluates G[s][t] once, loads the chunk's densities [s][r], and
// each thread accumulates 2 targets (t, t + 32) x 8 right-hand sides (r, r + 8, ...).
template <bool POLY>
__global__ void __launch_bounds__(256) k_p2p_b(const int32_t* __restrict__ leaf_start, const int4* __restrict__ leaf_ijk,
                                               const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr,
                                               const float4* __restrict__ pts, const float2* __restrict__ sig,
                                               float shift, int cap, int R, float2* __restrict__ phi) {
    constexpr float kC[HFMM_POLY_C_DEG + 1] = HFMM_POLY_C_INIT;
    constexpr float kS[HFMM_POLY_S_DEG + 1] = HFMM_POLY_S_INIT;
    extern __shared__ float4 smem_b[];
    const int cap4 = (cap + 3) & ~3;
    float4* sp = smem_b;                                      // [cap4] positions in the target leaf frame
    int* sj = reinterpret_cast<int*>(sp + cap4);              // [cap4] sorted index of each staged source
    float2* G = reinterpret_cast<float2*>(sj + cap4);         // [kBChunk][64]
    float2* Sg = G + kBChunk * 64;                            // [kBChunk][kBMax]
    __shared__ NbrTable T;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tid < 32) build_nbr_table(b, leaf_start, leaf_ijk, nbr_ptr, nbr, shift, false, T);
    __syncthreads();
    const int total = T.off[T.nl];
    for (int p = tid; p < total; p += blockDim.x) {  // one flat pass: loads of all leaves in flight
        const int q = nbr_segment(T, p);
        const int j = T.j0[q] + (p - T.off[q]);
        const float4 pt = __ldg(pts + j);
        const float4 o = T.sh[q];
        sp[p] = make_float4(pt.x + o.x, pt.y + o.y, pt.z + o.z, 0.f);
        sj[p] = j;
    }
    __syncthreads();  // staged positions and indices visible
    const int nself = T.cnt[0], out0 = __ldg(leaf_start + b);
    // thread (tt, rg): targets tt + 16a (a < 2, or < 4 for more than 32 targets), right-hand
    // sides rg + 16q (q < 4); per source 2-4 G loads and 4 density loads for 8-16 complex MACs
    const int tt = tid & 15, rg = tid >> 4;
    constexpr int kPre = kBChunk * kBMax / 256;  // densities per thread per chunk
    for (int t0 = 0; t0 < nself; t0 += 64) {
        const int nt = min(64, nself - t0);
        const bool two = nt > 32;  // uniform over the block
        float2 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);
        float2 pre[kPre];
        auto fetch = [&](int s0) {
            const int cnt = min(kBChunk, total - s0);
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int e = tid + 256 * q, s = e / kBMax, r = e % kBMax;
                pre[q] = (s < cnt && r < R) ? __ldg(sig + (int64_t)sj[s0 + s] * R + r) : make_float2(0.f, 0.f);
            }
        };
        fetch(0);
        for (int s0 = 0; s0 < total; s0 += kBChunk) {
            const int cnt = min(kBChunk, total - s0);
            __syncthreads();  // previous chunk consumed
            for (int e = tid; e < kBChunk * 64; e += 256) {
                const int s = e >> 6, t = e & 63;
                float2 g = make_float2(0.f, 0.f);
                const int si = s0 + s, ti = t0 + t;
                if (s < cnt && t < nt && si != ti) {  // si == ti: the target itself (self leaf first)
                    const float4 a = sp[si], c = sp[ti];
                    const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
                    const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float rinv = rsqrt_ftz(u);
                    if (POLY) {
                        g = make_float2(horner<HFMM_POLY_C_DEG>(kC, u) * rinv, horner<HFMM_POLY_S_DEG>(kS, u));
                    } else {
                        float sn, cs;
                        sincosf(u * rinv, &sn, &cs);
                        g = make_float2(cs * rinv, sn * rinv);
                    }
                }
                G[e] = g;
            }
#pragma unroll
            for (int q = 0; q < kPre; ++q) Sg[tid + 256 * q] = pre[q];
            __syncthreads();
            if (s0 + kBChunk < total) fetch(s0 + kBChunk);  // overlaps the multiply below
            for (int s = 0; s < cnt; ++s) {
                float2 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = Sg[s * kBMax + rg + 16 * q];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (a >= 2 && !two) break;
                    const float2 g = G[s * 64 + tt + 16 * a];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        acc[a][q].x = fmaf(g.x, v[q].x, fmaf(-g.y, v[q].y, acc[a][q].x));
                        acc[a][q].y = fmaf(g.x, v[q].y, fmaf(g.y, v[q].x, acc[a][q].y));
                    }
                }
            }
        }
        // potentials through shared memory (G and Sg are one 64 x 64 tile), then coalesced
        __syncthreads();
        float2* T = G;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) T[(tt + 16 * a) * kBMax + rg + 16 * q] = acc[a][q];
        __syncthreads();
        for (int e = tid; e < nt * R; e += 256) {
            const int t = e / R, r = e % R;
            phi[(int64_t)(out0 + t0) * R + e] = T[t * kBMax + r];
        }
    }
}

static size_t p2p_b_smem(int cap) {
    const size_t cap4 = (size_t)((cap + 3) & ~3);
    return cap4 * (sizeof(float4) + sizeof(int)) + sizeof(float2) * kBChunk * (64 + kBMax);
}

// M[leaf][r][c] = sum_j conj(b_c(y_j)) sig_b[j][r]; one block per leaf, 16 x 16 threads,
// 4 coefficients x 4 right-hand sides each, coefficient tiles of 64
template <int PP>
__global__ void __launch_bounds__(256) k_p2m_b(const int32_t* __restrict__ leaf_start, const float4* __restrict__ pts,
                                               const float2* __restrict__ sig, int p, float s, int R,
                                               float2* __restrict__ M) {
    extern __shared__ float2 smem_p2m[];
    const int P = (p + 1) * (p + 1);
    float2* Bs = smem_p2m;          // [kBChunk][P]
    float2* Ss = Bs + kBChunk * P;  // [kBChunk][kBMax]
    const int leaf = blockIdx.x, tid = threadIdx.x;
    const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    const int cg = tid & 15, rg = tid >> 4;
    for (int c0 = 0; c0 < P; c0 += 64) {
        float2 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);
        for (int j0 = b0; j0 < b1; j0 += kBChunk) {
            const int cnt = min(kBChunk, b1 - j0);
            __syncthreads();
            if (tid < cnt) regular_basis<PP>(pts[j0 + tid], p, s, Bs + tid * P);
            for (int e = tid; e < kBChunk * kBMax; e += 256) {
                const int j = e / kBMax, r = e % kBMax;
                Ss[e] = (j < cnt && r < R) ? sig[(int64_t)(j0 + j) * R + r] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int j = 0; j < cnt; ++j) {
                float2 bb[4], v[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int c = c0 + cg + 16 * a;
                    bb[a] = c < P ? Bs[j * P + c] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = Ss[j * kBMax + rg + 16 * q];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {  // conj(b) v
                        acc[a][q].x = fmaf(bb[a].x, v[q].x, fmaf(bb[a].y, v[q].y, acc[a][q].x));
                        acc[a][q].y = fmaf(bb[a].x, v[q].y, fmaf(-bb[a].y, v[q].x, acc[a][q].y));
                    }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + cg + 16 * a, r = rg + 16 * q;
                if (c < P && r < R) M[((int64_t)leaf * R + r) * P + c] = acc[a][q];
            }
    }
}

static size_t p2m_b_smem(int P) { return sizeof(float2) * kBChunk * (P + kBMax); }

// f(std::integral_constant<int, PP>) with PP = p for the fixed orders, -1 above them
template <typename F>
static void with_leaf_order(int p, F&& f) {
    switch (p) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        case 6: f(std::integral_constant<int, 6>{}); break;
        case 7: f(std::integral_constant<int, 7>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        default: f(std::integral_constant<int, -1>{}); break;
    }
}

// phi_b[j][r] += sum_c b_c(y_j) L[leaf][r][c]; one block per leaf; thread (point jj, rhs rg + 8q).
// A chunk's sums pass through shared memory (the basis buffer, rows of kBMax + 1) so that
// the read-modify-write of phi_b runs along r, contiguous in memory.
template <int PP>
__global__ void __launch_bounds__(256) k_l2p_b(const int32_t* __restrict__ leaf_start, const float4* __restrict__ pts,
                                               int p, float s, int R, const float2* __restrict__ L,
                                               float2* __restrict__ phi) {
    extern __shared__ float2 smem_l2p[];
    const int P = (p + 1) * (p + 1), Pp = P + 1;
    float2* Ls = smem_l2p;          // [kBMax][P]
    float2* Bs = Ls + kBMax * P;    // [kBChunk][P + 1], then the chunk's sums [kBChunk][kBMax + 1]
    const int leaf = blockIdx.x, tid = threadIdx.x;
    const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    for (int e = tid; e < kBMax * P; e += 256)
        Ls[e] = e < R * P ? L[(int64_t)leaf * R * P + e] : make_float2(0.f, 0.f);
    const int jj = tid & 31, rg = tid >> 5;
    for (int j0 = b0; j0 < b1; j0 += kBChunk) {
        const int cnt = min(kBChunk, b1 - j0);
        __syncthreads();
        if (tid < cnt) regular_basis<PP>(pts[j0 + tid], p, s, Bs + tid * Pp);
        __syncthreads();
        float2 acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
        if (jj < cnt)
            for (int c = 0; c < P; ++c) {
                const float2 bb = Bs[jj * Pp + c];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 l = Ls[(rg + 8 * q) * P + c];
                    acc[q].x = fmaf(bb.x, l.x, fmaf(-bb.y, l.y, acc[q].x));
                    acc[q].y = fmaf(bb.x, l.y, fmaf(bb.y, l.x, acc[q].y));
                }
            }
        __syncthreads();  // the basis is read: its buffer takes the sums
        float2* Ts = Bs;
        if (jj < cnt)
#pragma unroll
            for (int q = 0; q < 8; ++q) Ts[jj * (kBMax + 1) + rg + 8 * q] = acc[q];
        __syncthreads();
        for (int e = tid; e < cnt * R; e += 256) {
            const int j = e / R, r = e % R;
            float2* o = phi + (int64_t)(j0 + j) * R + r;
            const float2 v = *o, a = Ts[j * (kBMax + 1) + r];
            *o = make_float2(v.x + a.x, v.y + a.y);
        }
    }
}

static size_t l2p_b_smem(int P) {
    return sizeof(float2) * ((size_t)kBMax * P + (size_t)kBChunk * (size_t)std::max(P + 1, kBMax + 1));
}

// phi_b[i][r] += sum_nz C_i,col sig_b[col][r]: one warp per row, lanes on right-hand sides
__global__ void __launch_bounds__(256) k_corr_b(int64_t N, int R, const int64_t* __restrict__ ptr,
                                                const int32_t* __restrict__ col, const float2* __restrict__ val,
                                                const float2* __restrict__ sig, float2* __restrict__ phi) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
        const float2 c = __ldg(val + q);
        const float2* sg = sig + (int64_t)__ldg(col + q) * R;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = lane + 32 * h;
            if (r < R) {
                const float2 v = __ldg(sg + r);
                acc[h].x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc[h].x));
                acc[h].y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc[h].y));
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        if (r < R) {
            float2* o = phi + i * R + r;
            const float2 v = *o;
            *o = make_float2(v.x + acc[h].x, v.y + acc[h].y);
        }
    }
}

bool batch_supported(const hfmm_plan* P, int R) {
    if (R < 2 || R > kBMax || P->adaptive) return false;
    if (P->L >= 2 && P->lev[P->L].P > kBMaxP) return false;
    return P->p2p_cap > 0 && p2p_b_smem(P->p2p_cap) <= 200 * 1024;
}

// Once per device: the batched kernels may take up to the device's opt-in shared memory per
// block (each launch asks for what its plan needs).  A function's limit is process-wide, so a
// per-plan value would let a plan with a smaller neighbourhood lower it under another plan's
// launch on another thread.
static void batch_kernels_init() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return;
    int optin = 0;
    HFMM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto allow = [&](const void* fn) {
        cudaFuncAttributes fa{};
        HFMM_CUDA(cudaFuncGetAttributes(&fa, fn));
        HFMM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    };
    allow((const void*)k_p2p_b<true>);
    allow((const void*)k_p2p_b<false>);
    allow((const void*)k_p2m_b<-1>);
    for (int p = 0; p <= 9; ++p)
        with_leaf_order(p, [&](auto pp) {
            constexpr int PP = decltype(pp)::value;
            allow((const void*)k_l2p_b<PP>);
        });
    if (dev >= 0 && dev < 64) done[dev] = true;
}

void batch_setup(hfmm_plan* P, int R, cudaStream_t st) {
    BatchState& B = P->batch;
    if (B.R == R && B.sig.p) return;
    if (B.graph) {
        HFMM_CUDA(cudaGraphExecDestroy(B.graph));
        B.graph = nullptr;
    }
    B.R = R;
    const int64_t N = P->N;
    size_t cnt = 0;
    B.sig.alloc((size_t)N * R, &cnt);
    B.phi.alloc((size_t)N * R, &cnt);
    B.coef.alloc((size_t)std::max<int64_t>(P->coef_total, 1) * R, &cnt);
    // one item per translation, R columns; offsets of the level arrays scale by R
    const auto& hi = P->host_items;
    std::vector<TransItem> items;
    std::vector<int64_t> start(hi.size() + 1, 0);
    for (size_t q = 0; q < hi.size(); ++q) {
        start[q] = (int64_t)items.size();
        for (int c = 0; c < hi[q].ncol; ++c) {
            TransItem t = hi[q];
            t.src = hi[q].src * R;
            t.dst = hi[q].dst * R;
            t.cols = hi[q].cols + c;
            t.ncol = (int16_t)R;
            items.push_back(t);
        }
    }
    start[hi.size()] = (int64_t)items.size();
    // M2L on the tensor cores: order the items by (level, tile of kTile target boxes, operator,
    // target) so that the blocks running at one time cover one tile of targets and all its
    // offsets; the tile's local expansions and its neighbourhood's multipoles (R times the
    // single right-hand-side sizes) then stay in L2 while they are reused.
    const int gmax = m2l_tc_max_group();
    std::vector<int4> groups;
    {
        constexpr int kTile = 256;
        struct Key {
            int64_t dst_base;
            int tile, opi;
            int32_t dst;
            int64_t item;
            int P;
        };
        std::vector<Key> keys;
        for (int64_t g = 0; g < P->n_tc_groups; ++g) {
            const int4 sg = P->host_groups[g];
            for (int64_t b = start[sg.x]; b < start[sg.x + sg.y]; ++b) {
                const int32_t dst = P->host_cols[items[b].cols].y;
                keys.push_back({items[b].dst, dst / kTile, sg.z, dst, b, sg.w});
            }
        }
        std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
            if (a.dst_base != b.dst_base) return a.dst_base < b.dst_base;
            if (a.tile != b.tile) return a.tile < b.tile;
            if (a.opi != b.opi) return a.opi < b.opi;
            return a.dst < b.dst;
        });
        // the M2L tensor-core items go first, in this order; the rest keep theirs
        std::vector<TransItem> tc_items;
        tc_items.reserve(keys.size());
        for (size_t q = 0; q < keys.size(); ++q) {
            tc_items.push_back(items[keys[q].item]);
            if (q == 0 || keys[q].dst_base != keys[q - 1].dst_base || keys[q].tile != keys[q - 1].tile ||
                keys[q].opi != keys[q - 1].opi || groups.back().y == gmax)
                groups.push_back(make_int4((int)q, 1, keys[q].opi, keys[q].P));
            else
                ++groups.back().y;
        }
        B.n_tc_m2l = (int64_t)groups.size();
        // append the remaining items after the reordered block, shifting every range
        const int64_t ntc = (int64_t)tc_items.size();
        std::vector<char> is_tc(items.size(), 0);
        for (const Key& k : keys) is_tc[k.item] = 1;
        std::vector<int64_t> remap(items.size() + 1, 0);
        int64_t pos = ntc;
        for (size_t q = 0; q < items.size(); ++q) {
            remap[q] = is_tc[q] ? -1 : pos;
            if (!is_tc[q]) {
                tc_items.push_back(items[q]);
                ++pos;
            }
        }
        remap[items.size()] = pos;
        // start[] maps single items to batched items; send non-M2L-tensor-core ranges through remap
        for (size_t q = 0; q < start.size(); ++q) {
            int64_t b = start[q];
            while (b < (int64_t)items.size() && is_tc[b]) ++b;  // a range never begins inside the M2L block
            start[q] = remap[b];
        }
        items.swap(tc_items);
    }
    const int L = P->L;
    B.m2m_items.assign(L + 2, {0, 0});
    B.l2l_items.assign(L + 2, {0, 0});
    for (int l = 0; l <= L && l < (int)P->m2m_items_begin.size(); ++l)
        B.m2m_items[l] = {start[P->m2m_items_begin[l]], start[P->m2m_items_end[l]]};
    for (int l = 0; l <= L && l < (int)P->l2l_items_begin.size(); ++l)
        B.l2l_items[l] = {start[P->l2l_items_begin[l]], start[P->l2l_items_end[l]]};
    B.m2l_simt.clear();
    for (const SimtRange& r : P->m2l_simt) B.m2l_simt.push_back({start[r.begin], start[r.end], r.pout_max, R});
    auto regroup = [&](int64_t g0, int64_t g1) {
        const int64_t before = (int64_t)groups.size();
        for (int64_t g = g0; g < g1; ++g) {
            const int4 sg = P->host_groups[g];
            for (int64_t b = start[sg.x]; b < start[sg.x + sg.y]; b += gmax)
                groups.push_back(make_int4((int)b, (int)std::min<int64_t>(gmax, start[sg.x + sg.y] - b), sg.z, sg.w));
        }
        return std::make_pair(before, (int64_t)groups.size());
    };
    B.m2m_tc.assign(L + 2, {0, 0});
    B.l2l_tc.assign(L + 2, {0, 0});
    for (int l = 0; l <= L && l < (int)P->m2m_tc.size(); ++l) B.m2m_tc[l] = regroup(P->m2m_tc[l].first, P->m2m_tc[l].second);
    for (int l = 0; l <= L && l < (int)P->l2l_tc.size(); ++l) B.l2l_tc[l] = regroup(P->l2l_tc[l].first, P->l2l_tc[l].second);
    B.items.upload(items, &cnt, st);
    B.tc_groups.upload(groups, &cnt, st);
    P->dev_bytes += cnt;
    // shared-memory limits above 48 KiB, set before any capture
    m2l_tc_init();
    batch_kernels_init();
}

void run_matvec_batched(hfmm_plan* P, const float2* density, float2* potential, cudaStream_t st) {
    BatchState& B = P->batch;
    const int64_t N = P->N;
    const int R = B.R;
    const unsigned nb32 = (unsigned)((N + 31) / 32);
    k_prep_b<<<nb32, 256, 0, st>>>(N, R, P->perm.p, P->wscale.p, density, B.sig.p);
    const size_t sp2p = p2p_b_smem(P->p2p_cap);
    if (P->poly_p2p)
        k_p2p_b<true><<<(unsigned)P->nleaf, 256, sp2p, st>>>(P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p,
                                                             P->pts.p, B.sig.p, P->p2p_shift, P->p2p_cap, R, B.phi.p);
    else
        k_p2p_b<false><<<(unsigned)P->nleaf, 256, sp2p, st>>>(P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p, P->nbr.p,
                                                              P->pts.p, B.sig.p, P->p2p_shift, P->p2p_cap, R, B.phi.p);
    P->launches += 2;
    const int L = P->L;
    if (L >= 2) {
        HFMM_CUDA(cudaMemsetAsync(B.coef.p, 0, sizeof(float2) * P->coef_total * R, st));
        const LevelInfo& lv = P->lev[L];
        k_p2m_b<-1><<<(unsigned)P->nleaf, 256, p2m_b_smem(lv.P), st>>>(P->leaf_start.p, P->pts.p, B.sig.p, lv.p,
                                                                      (float)lv.s, R, B.coef.p + lv.mofs * R);
        ++P->launches;
        for (int l = L - 1; l >= 2; --l) {
            const auto& g = B.m2m_tc[l];
            if (g.second > g.first) {
                m2l_tc_launch(B.tc_groups.p + g.first, g.second - g.first, B.items.p, P->item_cols.p, P->aops.p,
                              B.coef.p, P->dev_err.p, R, st);
                ++P->launches;
            } else {
                launch_translate(P, B.items.p, B.coef.p, R, B.m2m_items[l].first, B.m2m_items[l].second, P->lev[l].P,
                                 R, st);
            }
        }
        for (const SimtRange& r : B.m2l_simt)
            launch_translate(P, B.items.p, B.coef.p, R, r.begin, r.end, r.pout_max, r.width, st);
        if (B.n_tc_m2l > 0) {
            m2l_tc_launch(B.tc_groups.p, B.n_tc_m2l, B.items.p, P->item_cols.p, P->aops.p, B.coef.p, P->dev_err.p, R,
                          st);
            ++P->launches;
        }
        for (int l = 3; l <= L; ++l) {
            const auto& g = B.l2l_tc[l];
            if (g.second > g.first) {
                m2l_tc_launch(B.tc_groups.p + g.first, g.second - g.first, B.items.p, P->item_cols.p, P->aops.p,
                              B.coef.p, P->dev_err.p, R, st);
                ++P->launches;
            } else {
                launch_translate(P, B.items.p, B.coef.p, R, B.l2l_items[l].first, B.l2l_items[l].second, P->lev[l].P,
                                 R, st);
            }
        }
        with_leaf_order(lv.p, [&](auto pp) {
            k_l2p_b<decltype(pp)::value><<<(unsigned)P->nleaf, 256, l2p_b_smem(lv.P), st>>>(
                P->leaf_start.p, P->pts.p, lv.p, (float)lv.s, R, B.coef.p + lv.lofs * R, B.phi.p);
        });
        ++P->launches;
    }
    if (P->corr_nnz > 0) {
        k_corr_b<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(N, R, P->corr_ptr.p, P->corr_col.p, P->corr_val.p,
                                                                  B.sig.p, B.phi.p);
        ++P->launches;
    }
    k_output_b<<<nb32, 256, 0, st>>>(N, R, P->perm.p, B.phi.p, potential);
    ++P->launches;
    HFMM_CUDA(cudaGetLastError());
}

// R right-hand sides (2..64) in one batched matvec, replayed from a CUDA graph captured on
// the plan's own stream (the caller's stream may be the legacy default stream, which cannot
// be captured) and re-captured when the buffers change.
void batched_matvec(hfmm_plan* P, const float2* d, float2* o, int R, cudaStream_t st) {
    BatchState& B = P->batch;
    batch_setup(P, R, st);
    if (!B.cap_stream) HFMM_CUDA(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
    if (!B.graph || B.g_in != (const void*)d || B.g_out != (void*)o) {
        if (B.graph) {
            HFMM_CUDA(cudaGraphExecDestroy(B.graph));
            B.graph = nullptr;
        }
        const int64_t l0 = P->launches;
        if (!capture_graph(B.cap_stream, [&] { run_matvec_batched(P, d, o, B.cap_stream); }, &B.graph)) {
            P->launches = l0;  // the capture was invalidated (see capture_graph): run the matvec directly
            run_matvec_batched(P, d, o, st);
            return;
        }
        B.g_launches = P->launches - l0;
        P->launches = l0;
        B.g_in = d;
        B.g_out = o;
    }
    HFMM_CUDA(cudaGraphLaunch(B.graph, st));
    P->launches += B.g_launches;
}

// ============================================================== off-surface evaluation
// Sources staged as FP32 hi + lo positions (relative to the mesh's bounding-box centre) and
// the strength w sigma / (4 pi); a source-target difference (t_hi - s_hi) + (t_lo - s_lo) is
// then exact to ~1e-14 before the FP32 distance is formed.
__global__ void k_field_stage(int64_t N, const double* __restrict__ x64, const double* __restrict__ w,
                              const float2* __restrict__ density, double cx, double cy, double cz,
                              float4* __restrict__ hi, float4* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = x64[3 * i] - cx, y = x64[3 * i + 1] - cy, z = x64[3 * i + 2] - cz;
    const float xh = (float)x, yh = (float)y, zh = (float)z;
    const double sc = w[i] / (4.0 * 3.14159265358979323846);
    const float2 d = density[i];
    hi[i] = make_float4(xh, yh, zh, (float)(sc * d.x));
    lo[i] = make_float4((float)(x - xh), (float)(y - yh), (float)(z - zh), (float)(sc * d.y));
}

__global__ void __launch_bounds__(256) k_field(int64_t nt, const double* __restrict__ tg, double cx, double cy,
                                               double cz, int64_t N, const float4* __restrict__ hi,
                                               const float4* __restrict__ lo, float k, float2* __restrict__ out) {
    __shared__ float4 sh[256], sl[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float th[3] = {0.f, 0.f, 0.f}, tl[3] = {0.f, 0.f, 0.f};
    if (t < nt) {
        const double p[3] = {tg[3 * t] - cx, tg[3 * t + 1] - cy, tg[3 * t + 2] - cz};
        for (int d = 0; d < 3; ++d) {
            th[d] = (float)p[d];
            tl[d] = (float)(p[d] - (double)th[d]);
        }
    }
    float ar = 0.f, ai = 0.f;
    for (int64_t j0 = 0; j0 < N; j0 += 256) {
        const int64_t j = j0 + threadIdx.x;
        if (j < N) {
            sh[threadIdx.x] = hi[j];
            sl[threadIdx.x] = lo[j];
        }
        __syncthreads();
        const int cnt = (N - j0 < 256) ? (int)(N - j0) : 256;
        for (int q = 0; q < cnt; ++q) {
            const float4 a = sh[q], b = sl[q];
            const float dx = (th[0] - a.x) + (tl[0] - b.x);
            const float dy = (th[1] - a.y) + (tl[1] - b.y);
            const float dz = (th[2] - a.z) + (tl[2] - b.z);
            const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            float sn, cs;
            sincosf(k * r, &sn, &cs);
            const float ir = 1.f / r;
            const float re = cs * ir, im = sn * ir;
            ar = fmaf(a.w, re, fmaf(-b.w, im, ar));
            ai = fmaf(a.w, im, fmaf(b.w, re, ai));
        }
        __syncthreads();
    }
    if (t < nt) out[t] = make_float2(ar, ai);
}

void run_field(hfmm_plan* P, const float2* density, const double* targets, int64_t nt, float2* out,
               cudaStream_t st) {
    const int64_t N = P->N;
    if (!P->w_user.p) {
        P->w_user.upload(P->host_w, nullptr, st);
        P->fsrc_hi.alloc(N, nullptr);
        P->fsrc_lo.alloc(N, nullptr);
    }
    const double cx = P->lo[0] + 0.5 * P->D, cy = P->lo[1] + 0.5 * P->D, cz = P->lo[2] + 0.5 * P->D;
    k_field_stage<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, P->x64.p, P->w_user.p, density, cx, cy, cz,
                                                               P->fsrc_hi.p, P->fsrc_lo.p);
    if (nt > 0)
        k_field<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, targets, cx, cy, cz, N, P->fsrc_hi.p,
                                                              P->fsrc_lo.p, (float)P->k, out);
    P->launches += 2;
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
