// FMM matvec kernels (FP32) for the Helmholtz single-layer operator.
//
// One matvec (Sec. 2.3 and the Nystrom operator of Sec. 2.2):
//   density prep   sh_i = k w_i s_perm(i) / (4 pi)  (Morton order)
//   near field     phi_i  = sum_{j in neighbour leaves, j != i} sh_j (C(u)/sqrt(u) + i S(u)),
//                  u = (k R_ij)^2   [= w_j s_j exp(ikR)/(4 pi R), Eq. 6; Listing 1's P2P]
//   far field      P2M -> M2M -> M2L -> L2L -> L2P   (Eq. 11-14)
//   correction     phi_i += sum_j C~_ij sh_j  (exact self/near integrals minus point terms)
//   output         potential[perm(i)] = phi_i
#include <algorithm>
#include <cmath>

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
    T o;
    o.x = v.x;
    o.y = v.y;
    out[perm[i]] = o;
}

void launch_density_prep(hfmm_plan* P, const void* density, bool fp64, float2* sig, cudaStream_t st) {
    ++P->launches;
    unsigned nb = (unsigned)((P->N + 255) / 256);
    if (fp64)
        k_density_prep<double2><<<nb, 256, 0, st>>>(P->N, P->perm.p, P->wscale.p, (const double2*)density, sig);
    else
        k_density_prep<float2><<<nb, 256, 0, st>>>(P->N, P->perm.p, P->wscale.p, (const float2*)density, sig);
}

void launch_output(hfmm_plan* P, const float2* phi, void* out, bool fp64, cudaStream_t st) {
    ++P->launches;
    unsigned nb = (unsigned)((P->N + 255) / 256);
    if (fp64) k_output<double2><<<nb, 256, 0, st>>>(P->N, P->perm.p, phi, (double2*)out);
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

// Accumulates the interactions of one target with the points [j0, j1) of one
// source leaf.  (tx,ty,tz): target relative to the source leaf centre, scaled by k.
template <bool POLY, bool MASK>
__device__ __forceinline__ void p2p_leaf(float tx, float ty, float tz, int32_t j0, int32_t j1, int32_t self_i,
                                         const float4* __restrict__ pts, const float2* __restrict__ sig,
                                         float& ar, float& ai) {
    constexpr float kC[HFMM_POLY_C_DEG + 1] = HFMM_POLY_C_INIT;
    constexpr float kS[HFMM_POLY_S_DEG + 1] = HFMM_POLY_S_INIT;
#pragma unroll 4
    for (int32_t j = j0; j < j1; ++j) {
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

// One warp per target tile (<= 32 points of one leaf); lanes own targets,
// sources are read with warp-uniform (broadcast) loads.
template <bool POLY>
__global__ void __launch_bounds__(128) k_p2p(int64_t ntiles, const int4* __restrict__ tiles,
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
    bool active = lane < tl.z;
    int32_t i = tl.y + (active ? lane : 0);
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
        int32_t j0 = __ldg(leaf_start + s), j1 = __ldg(leaf_start + s + 1);
        if (s == leaf) p2p_leaf<POLY, true>(tx, ty, tz, j0, j1, i, pts, sig, ar, ai);
        else p2p_leaf<POLY, false>(tx, ty, tz, j0, j1, i, pts, sig, ar, ai);
    }
    if (active) phi[i] = make_float2(ar, ai);
}

// ============================================================== FP32 special functions
// out[n] = j_n(x) / s^n, n = 0..p
__device__ static void f_jn_scaled(int p, float x, float s, float* out) {
    if (x < 2.0f) {
        float lead = 1.0f, xs = x / s, h = -0.5f * x * x;
        for (int n = 0; n <= p; ++n) {
            if (n) lead *= xs / (float)(2 * n + 1);
            float term = 1.0f, sum = 1.0f;
            for (int q = 1; q < 24; ++q) {
                term *= h / (float)(q * (2 * n + 2 * q + 1));
                sum += term;
                if (fabsf(term) < 1e-8f * fabsf(sum)) break;
            }
            out[n] = lead * sum;
        }
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

// ============================================================== P2M
// One block per leaf.  Points are staged in chunks: each staged point stores
// jt_n Q_n^m (m >= 0, triangular index) and sh e^{-i m phi}, sh e^{+i m phi}.
__global__ void k_p2m(const int32_t* __restrict__ leaf_start, const float4* __restrict__ pts,
                      const float2* __restrict__ sig, int p, float s, int chunk, float2* __restrict__ M) {
    extern __shared__ float sm[];
    int leaf = blockIdx.x;
    int P = (p + 1) * (p + 1);
    int H = (p + 1) * (p + 2) / 2;
    int stride = H + 4 * (p + 1);
    int32_t b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    for (int c0 = 0; c0 < P; c0 += blockDim.x) {
        int c = c0 + threadIdx.x;
        int n = 0, m = 0;
        if (c < P) {
            n = (int)sqrtf((float)c);
            while (n * n > c) --n;
            while ((n + 1) * (n + 1) <= c) ++n;
            m = c - n * n - n;
        }
        int hidx = n * (n + 1) / 2 + (m < 0 ? -m : m);
        float accr = 0.f, acci = 0.f;
        for (int32_t j0 = b0; j0 < b1; j0 += chunk) {
            int cnt = min(chunk, b1 - j0);
            if (threadIdx.x < cnt) {
                float* row = sm + threadIdx.x * stride;
                float4 y = pts[j0 + threadIdx.x];
                float2 sg = sig[j0 + threadIdx.x];
                Dir d = make_dir(y.x, y.y, y.z);
                float jr[HFMM_PMAX + 1];
                f_jn_scaled(p, d.r, s, jr);
                float qmm = 0.28209479177387814f;
                float er = 1.f, ei = 0.f;
                for (int mm = 0; mm <= p; ++mm) {
                    if (mm > 0) {
                        qmm *= sqrtf((2.f * mm + 1.f) / (2.f * mm)) * d.st;
                        float t = er * d.ex - ei * d.ey;
                        ei = er * d.ey + ei * d.ex;
                        er = t;
                    }
                    // sh e^{-i m phi} and sh e^{+i m phi}
                    row[H + 4 * mm + 0] = sg.x * er + sg.y * ei;
                    row[H + 4 * mm + 1] = sg.y * er - sg.x * ei;
                    row[H + 4 * mm + 2] = sg.x * er - sg.y * ei;
                    row[H + 4 * mm + 3] = sg.y * er + sg.x * ei;
                    float qa = qmm, qb = 0.f;
                    for (int nn = mm; nn <= p; ++nn) {
                        float qn;
                        if (nn == mm) qn = qmm;
                        else if (nn == mm + 1) qn = sqrtf(2.f * mm + 3.f) * d.ct * qmm;
                        else {
                            float a = sqrtf((4.f * nn * nn - 1.f) / (float)(nn * nn - mm * mm));
                            float bb = sqrtf((float)((nn - 1) * (nn - 1) - mm * mm) / (4.f * (nn - 1) * (nn - 1) - 1.f));
                            qn = a * (d.ct * qa - bb * qb);
                        }
                        if (nn > mm) { qb = qa; qa = qn; }
                        row[nn * (nn + 1) / 2 + mm] = jr[nn] * qn;
                    }
                }
            }
            __syncthreads();
            if (c < P) {
                int eo = H + 4 * (m < 0 ? -m : m) + (m < 0 ? 2 : 0);
                for (int t = 0; t < cnt; ++t) {
                    const float* row = sm + t * stride;
                    float b = row[hidx];
                    accr = fmaf(b, row[eo], accr);
                    acci = fmaf(b, row[eo + 1], acci);
                }
            }
            __syncthreads();
        }
        if (c < P) M[(int64_t)leaf * P + c] = make_float2(accr, acci);
    }
}

// ============================================================== L2P
__global__ void k_l2p(int64_t N, const int32_t* __restrict__ pt_leaf, const float4* __restrict__ pts, int p,
                      float s, const float2* __restrict__ Lc, float2* __restrict__ phi) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int P = (p + 1) * (p + 1);
    const float2* L = Lc + (int64_t)pt_leaf[i] * P;
    float4 y = pts[i];
    Dir d = make_dir(y.x, y.y, y.z);
    float jr[HFMM_PMAX + 1];
    f_jn_scaled(p, d.r, s, jr);
    float accr = 0.f, acci = 0.f;
    float qmm = 0.28209479177387814f;
    float er = 1.f, ei = 0.f;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            qmm *= sqrtf((2.f * m + 1.f) / (2.f * m)) * d.st;
            float t = er * d.ex - ei * d.ey;
            ei = er * d.ey + ei * d.ex;
            er = t;
        }
        float qa = qmm, qb = 0.f;
        for (int n = m; n <= p; ++n) {
            float qn;
            if (n == m) qn = qmm;
            else if (n == m + 1) qn = sqrtf(2.f * m + 3.f) * d.ct * qmm;
            else {
                float a = sqrtf((4.f * n * n - 1.f) / (float)(n * n - m * m));
                float bb = sqrtf((float)((n - 1) * (n - 1) - m * m) / (4.f * (n - 1) * (n - 1) - 1.f));
                qn = a * (d.ct * qa - bb * qb);
            }
            if (n > m) { qb = qa; qa = qn; }
            float b = jr[n] * qn;
            float2 lp = L[n * n + n + m];
            // L_{n,m} b e^{+i m phi}
            accr += b * (lp.x * er - lp.y * ei);
            acci += b * (lp.x * ei + lp.y * er);
            if (m > 0) {
                float2 lm = L[n * n + n - m];
                accr += b * (lm.x * er + lm.y * ei);
                acci += b * (lm.y * er - lm.x * ei);
            }
        }
    }
    float2 o = phi[i];
    phi[i] = make_float2(o.x + accr, o.y + acci);
}

// ============================================================== batched translations
// Out[:, dst] += T * In[:, src] for the column pairs of one work item.
// 128 threads, 32-row x 64-column output tiles, K in slices of 32.
__global__ void __launch_bounds__(128) k_translate(const TransItem* __restrict__ items, int64_t item0,
                                                   const int2* __restrict__ cols, const float2* __restrict__ ops,
                                                   float2* __restrict__ coef) {
    __shared__ float2 sT[32][33];
    __shared__ float2 sX[32][65];
    __shared__ int2 sc[HFMM_TRANS_NB];
    TransItem it = items[item0 + blockIdx.x];
    int tid = threadIdx.x;
    int ncol = it.ncol, Pin = it.pin, Pout = it.pout;
    if (tid < HFMM_TRANS_NB) sc[tid] = tid < ncol ? cols[it.cols + tid] : make_int2(0, 0);
    __syncthreads();
    const float2* T = ops + it.op;
    int tx = tid & 15, ty = tid >> 4;  // 16 column groups x 8 row groups
    for (int r0 = 0; r0 < Pout; r0 += 32) {
        float accr[4][4], acci[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) accr[a][b] = acci[a][b] = 0.f;
        for (int k0 = 0; k0 < Pin; k0 += 32) {
            // T tile: rows r0..r0+31, cols k0..k0+31
            for (int e = tid; e < 32 * 32; e += 128) {
                int rr = e >> 5, kk = e & 31;
                int r = r0 + rr, kq = k0 + kk;
                sT[rr][kk] = (r < Pout && kq < Pin) ? __ldg(T + (int64_t)r * Pin + kq) : make_float2(0.f, 0.f);
            }
            // X tile: rows k0..k0+31 of the gathered source columns
            for (int e = tid; e < 32 * HFMM_TRANS_NB; e += 128) {
                int cc = e >> 5, kk = e & 31;
                int kq = k0 + kk;
                sX[kk][cc] = (cc < ncol && kq < Pin) ? __ldg(coef + it.src + (int64_t)sc[cc].x * Pin + kq)
                                                     : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < 32; ++kk) {
                float2 a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = sT[ty + 8 * q][kk];
                    b[q] = sX[kk][tx + 16 * q];
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
            int r = r0 + ty + 8 * qa;
            if (r >= Pout) continue;
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) {
                int cc = tx + 16 * qb;
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
}

// ============================================================== correction (CSR SpMV)
__global__ void k_corr(int64_t N, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                       const float2* __restrict__ val, const float2* __restrict__ sig, float2* __restrict__ phi) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= N) return;
    int64_t e0 = ptr[row], e1 = ptr[row + 1];
    float ar = 0.f, ai = 0.f;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        float2 v = __ldg(val + e);
        float2 s = __ldg(sig + __ldg(col + e));
        ar = fmaf(v.x, s.x, fmaf(-v.y, s.y, ar));
        ai = fmaf(v.x, s.y, fmaf(v.y, s.x, ai));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
        float2 v = phi[row];
        phi[row] = make_float2(v.x + ar, v.y + ai);
    }
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

static void launch_translate(hfmm_plan* P, int64_t b, int64_t e, cudaStream_t st) {
    if (e <= b) return;
    k_translate<<<(unsigned)(e - b), 128, 0, st>>>(P->items.p, b, P->item_cols.p, P->ops.p, P->coef.p);
    ++P->launches;
}

void run_matvec_sorted(hfmm_plan* P, int parts, cudaStream_t st) {
    int64_t N = P->N;
    mark_stage(P, 1, st);
    if (parts & 1) {
        unsigned nb = (unsigned)((P->ntiles * 32 + 127) / 128);
        if (P->poly_p2p)
            k_p2p<true><<<nb, 128, 0, st>>>(P->ntiles, P->tiles.p, P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p,
                                            P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift, P->phi.p);
        else
            k_p2p<false><<<nb, 128, 0, st>>>(P->ntiles, P->tiles.p, P->leaf_start.p, P->leaf_ijk.p, P->nbr_ptr.p,
                                             P->nbr.p, P->pts.p, P->sig.p, P->p2p_shift, P->phi.p);
        ++P->launches;
    } else {
        HFMM_CUDA(cudaMemsetAsync(P->phi.p, 0, sizeof(float2) * N, st));
    }
    mark_stage(P, 2, st);
    int L = P->L;
    bool far = (parts & 2) && L >= 2;
    if (far) {
        // multipoles above the leaves and all locals accumulate: clear them
        HFMM_CUDA(cudaMemsetAsync(P->coef.p, 0, sizeof(float2) * P->coef_total, st));
        const LevelInfo& lv = P->lev[L];
        int p = lv.p;
        int H = (p + 1) * (p + 2) / 2, stride = H + 4 * (p + 1);
        int chunk = std::max(1, std::min(32, (40 * 1024) / (stride * 4)));
        k_p2m<<<(unsigned)P->nleaf, 128, (size_t)chunk * stride * sizeof(float), st>>>(
            P->leaf_start.p, P->pts.p, P->sig.p, p, (float)lv.s, chunk, P->coef.p + lv.mofs);
        ++P->launches;
    }
    mark_stage(P, 3, st);
    if (far)
        for (int l = L - 1; l >= 2; --l) launch_translate(P, P->m2m_items_begin[l], P->m2m_items_end[l], st);
    mark_stage(P, 4, st);
    if (far) {
        for (const auto& r : P->m2l_simt_ranges) launch_translate(P, r.first, r.second, st);
        if (P->n_tc_groups > 0) {
            m2l_tc_launch(P->tc_groups.p, P->n_tc_groups, P->items.p, P->item_cols.p, P->aops.p, P->coef.p,
                          P->dev_err.p, st);
            ++P->launches;
        }
    }
    mark_stage(P, 5, st);
    if (far)
        for (int l = 3; l <= L; ++l) launch_translate(P, P->l2l_items_begin[l], P->l2l_items_end[l], st);
    mark_stage(P, 6, st);
    if (far) {
        const LevelInfo& lv = P->lev[L];
        k_l2p<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(N, P->pt_leaf.p, P->pts.p, lv.p, (float)lv.s,
                                                           P->coef.p + lv.lofs, P->phi.p);
        ++P->launches;
    }
    mark_stage(P, 7, st);
    if ((parts & 4) && P->corr_nnz > 0) {
        k_corr<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(N, P->corr_ptr.p, P->corr_col.p, P->corr_val.p,
                                                               P->sig.p, P->phi.p);
        ++P->launches;
    }
    mark_stage(P, 8, st);
    HFMM_CUDA(cudaGetLastError());
}

void run_direct_sorted(hfmm_plan* P, cudaStream_t st) {
    int64_t N = P->N;
    k_direct<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, P->pts.p, P->pt_leaf.p, P->leaf_ijk.p, P->sig.p,
                                                          P->p2p_shift, P->phi.p);
    ++P->launches;
    if (P->corr_nnz > 0) {
        k_corr<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(N, P->corr_ptr.p, P->corr_col.p, P->corr_val.p,
                                                               P->sig.p, P->phi.p);
        ++P->launches;
    }
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
