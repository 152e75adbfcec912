// Restarted GMRES(m) on the device (the paper's solver: GMRES with the FMM as
// the matvec, exit at a relative residual of 1e-4; Sec. 1, 5.1, 6.4).
//
// Precision.  The Krylov basis, the work vector, the iterate and the
// right-hand side are double-float complex vectors: each real value is an
// unevaluated sum hi + lo of two FP32 numbers (48-bit significand), stored as
// float4 (re_hi, im_hi, re_lo, im_lo), the same 16 bytes per element as FP64
// complex.  The element-wise Arnoldi work (Gram-Schmidt inner products and
// updates, norms, scaling, the solution update) runs on the FP32 pipe with
// error-free transformations: the exact product error of an FMA (TwoProd),
// Knuth's TwoSum, and the compensated dot product of Ogita, Rump and Oishi
// (Dot2), which returns a sum as accurate as if it were accumulated in twice
// the working precision.  This keeps the orthogonalisation FP64-class
// (relative errors near 2^-48) while the FP32 pipe, about 70 times faster than
// this GPU's FP64 pipe, leaves the kernels bound by HBM.  Per-block partial
// sums are combined in FP64.  For one right-hand side the Gram-Schmidt
// coefficients, the (m+1) x m Hessenberg matrix, its Givens rotations and the
// triangular solve stay on the device in FP64 (single-thread kernels), and the
// host reads one residual estimate per iteration; the lockstep solver for several
// right-hand sides keeps them on the host.  The matvec is the FP32 FMM.
#include <cmath>
#include <complex>
#include <vector>

#include "hfmm_internal.cuh"

namespace hfmm {

using cd = std::complex<double>;

// The host waits for `st` through a blocking-sync event: the thread sleeps instead of spinning,
// so that many solves in flight (one host thread each, as in serving) leave the host cores to
// the plan builds and launches beside them.
static void host_wait(hfmm_plan* P, cudaStream_t st) {
    if (!P->host_ev) HFMM_CUDA(cudaEventCreateWithFlags(&P->host_ev, cudaEventBlockingSync | cudaEventDisableTiming));
    HFMM_CUDA(cudaEventRecord(P->host_ev, st));
    HFMM_CUDA(cudaEventSynchronize(P->host_ev));
}

static constexpr int RB = 256;  // threads per reduction block
static constexpr int RG = 296;  // reduction blocks per vector (2 per SM)
static constexpr int kDotVecs = 8;  // basis vectors per inner-product block (w is read once per 8)

// ------------------------------------------------------------ error-free transformations
// Every operation is an explicit round-to-nearest intrinsic, so nothing is fused or reassociated.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b| or a = 0
    s = __fadd_rn(a, b);
    e = __fadd_rn(b, -__fadd_rn(s, -a));
}

// Dot2 accumulator: the value is s + c (s carries the running sum, c its error terms).
struct Acc {
    float s = 0.f, c = 0.f;
    // += (ah + al)(bh + bl); the al*bl term (relative size 2^-48) is dropped
    __device__ __forceinline__ void add_prod(float ah, float al, float bh, float bl) {
        const float p = __fmul_rn(ah, bh);
        float q = __fmaf_rn(ah, bh, -p);  // exact: ah bh = p + q
        q = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, q));
        float t, r;
        two_sum(s, p, t, r);
        s = t;
        c = __fadd_rn(c, __fadd_rn(q, r));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// (ah + al) + (bh + bl), renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, h, l);
}

// a double as hi + lo (host side)
static inline void split_df(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// ------------------------------------------------------------ element-wise kernels
__global__ void k_c64_to_df(int64_t N, const float2* __restrict__ a, float4* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_float4(a[i].x, a[i].y, 0.f, 0.f);
}
__global__ void k_df_to_c64(int64_t N, const float4* __restrict__ a, float2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_float2(a[i].x, a[i].y);  // hi = round(hi + lo) for a normalised pair
}
// b = s a with s = sh + sl
__global__ void k_scale_df(int64_t N, const float4* __restrict__ a, float sh, float sl, float4* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 v = a[i];
    float4 o;
    {
        const float p = __fmul_rn(v.x, sh);
        const float q = __fmaf_rn(v.x, sl, __fmaf_rn(v.z, sh, __fmaf_rn(v.x, sh, -p)));
        fast_two_sum(p, q, o.x, o.z);
    }
    {
        const float p = __fmul_rn(v.y, sh);
        const float q = __fmaf_rn(v.y, sl, __fmaf_rn(v.w, sh, __fmaf_rn(v.y, sh, -p)));
        fast_two_sum(p, q, o.y, o.w);
    }
    b[i] = o;
}
// c = a - b
__global__ void k_sub_df(int64_t N, const float4* __restrict__ a, const float4* __restrict__ b,
                         float4* __restrict__ c) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 u = a[i], v = b[i];
    float4 o;
    df_add(u.x, u.z, -v.x, -v.z, o.x, o.z);
    df_add(u.y, u.w, -v.y, -v.w, o.y, o.w);
    c[i] = o;
}

// block-wide FP64 sum of a complex value (thread 0 gets it)
__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double2 r = make_double2(0, 0);
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            r.x += sh[q].x;
            r.y += sh[q].y;
        }
    __syncthreads();
    return r;
}

// partial[i * RG + blk] = sum over the block's rows of conj(V_i) w, for the kDotVecs vectors
// i = blockIdx.y * kDotVecs + c (< nvec); grid RG x ceil(nvec / kDotVecs).  with_norm: the
// blocks of y = 0 also leave |w|^2 in partial[nvec * RG + blk].  skip (may be NULL): when *skip
// is set the pass is not needed and the kernel returns at once.
__global__ void __launch_bounds__(RB, 2) k_dots_df(int64_t N, const float4* __restrict__ V, int nvec,
                                                const float4* __restrict__ w, double2* __restrict__ partial,
                                                const int* __restrict__ skip, int with_norm,
                                                const int* __restrict__ jd = nullptr) {
    if (skip && *skip) return;
    if (jd) nvec = *jd + 1;  // the iteration index held on the device (graph-replayed steps)
    __shared__ double2 sh[RB / 32];
    const int i0 = blockIdx.y * kDotVecs;
    if (i0 >= nvec) return;  // uniform over the block (grids sized for the longest step)
    const int nv = min(kDotVecs, nvec - i0);
    const bool nrm = with_norm && blockIdx.y == 0;
    Acc re[kDotVecs], im[kDotVecs], wn;
    for (int64_t r = (int64_t)blockIdx.x * RB + threadIdx.x; r < N; r += (int64_t)RG * RB) {
        const float4 b = w[r];
        if (nrm) {
            wn.add_prod(b.x, b.z, b.x, b.z);
            wn.add_prod(b.y, b.w, b.y, b.w);
        }
        // all the row's loads in flight before the arithmetic (absent vectors read as zero,
        // which adds nothing)
        float4 av[kDotVecs];
#pragma unroll
        for (int c = 0; c < kDotVecs; ++c)
            av[c] = c < nv ? V[(int64_t)(i0 + c) * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kDotVecs; ++c) {
            const float4 a = av[c];
            // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
            re[c].add_prod(a.x, a.z, b.x, b.z);
            re[c].add_prod(a.y, a.w, b.y, b.w);
            im[c].add_prod(a.x, a.z, b.y, b.w);
            im[c].add_prod(-a.y, -a.w, b.x, b.z);
        }
    }
#pragma unroll
    for (int c = 0; c < kDotVecs; ++c) {
        if (c >= nv) break;  // uniform over the block
        const double2 s = block_sum2(make_double2(re[c].value(), im[c].value()), sh);
        if (threadIdx.x == 0) partial[(int64_t)(i0 + c) * RG + blockIdx.x] = s;
    }
    if (nrm) {  // uniform over the block
        const double2 s = block_sum2(make_double2(wn.value(), 0.0), sh);
        if (threadIdx.x == 0) partial[(int64_t)nvec * RG + blockIdx.x] = s;
    }
}

// partial[blk] = sum |w|^2 over the block's rows
__global__ void __launch_bounds__(RB) k_norm2_df(int64_t N, const float4* __restrict__ w,
                                                 double2* __restrict__ partial) {
    __shared__ double2 sh[RB / 32];
    Acc a;
    for (int64_t r = (int64_t)blockIdx.x * RB + threadIdx.x; r < N; r += (int64_t)RG * RB) {
        const float4 b = w[r];
        a.add_prod(b.x, b.z, b.x, b.z);
        a.add_prod(b.y, b.w, b.y, b.w);
    }
    const double2 s = block_sum2(make_double2(a.value(), 0.0), sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[i] = sum_b partial[i * RG + b]   (one block per vector, FP64)
__global__ void __launch_bounds__(RB) k_reduce(const double2* __restrict__ partial, double2* __restrict__ out) {
    __shared__ double2 sh[RB / 32];
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < RG; b += RB) {
        double2 v = partial[(int64_t)blockIdx.x * RG + b];
        acc.x += v.x;
        acc.y += v.y;
    }
    double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// x += sign * sum_i h_i V_i, with h given as double-float pairs hdf[i] = (re_hi, im_hi, re_lo, im_lo)
__global__ void k_axpy_df(int64_t N, const float4* __restrict__ V, int nvec, const float4* __restrict__ hdf,
                          float sign, float4* __restrict__ x, const int* __restrict__ skip = nullptr,
                          const int* __restrict__ jd = nullptr) {
    if (skip && *skip) return;
    if (jd) nvec = *jd + 1;
    extern __shared__ float4 hs[];
    for (int q = threadIdx.x; q < nvec; q += blockDim.x) hs[q] = hdf[q];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    Acc ar, ai;
    for (int i = 0; i < nvec; ++i) {
        const float4 a = V[(int64_t)i * N + r], h = hs[i];
        // h a = (hr ar - hi ai) + i (hr ai + hi ar)
        ar.add_prod(h.x, h.z, a.x, a.z);
        ar.add_prod(-h.y, -h.w, a.y, a.w);
        ai.add_prod(h.x, h.z, a.y, a.w);
        ai.add_prod(h.y, h.w, a.x, a.z);
    }
    float4 o = x[r];
    float sh, sl;
    two_sum(ar.s, ar.c, sh, sl);
    df_add(o.x, o.z, sign * sh, sign * sl, o.x, o.z);
    two_sum(ai.s, ai.c, sh, sl);
    df_add(o.y, o.w, sign * sh, sign * sl, o.y, o.w);
    x[r] = o;
}

// ------------------------------------------------------------ device-side Arnoldi bookkeeping
// The Hessenberg column, the Givens rotations, the least-squares right-hand side and the
// triangular solve live in device memory (FP64); the host reads one residual estimate per
// iteration instead of every coefficient.

__device__ __forceinline__ float4 to_df4(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

// block i: h_i = sum of its RG partials; coeff[i] = h_i as double-float (the update
// w -= V h); hsum[i] += h_i (the Hessenberg column, summed over the two passes)
__global__ void __launch_bounds__(RB) k_reduce_h(const double2* __restrict__ partial, float4* __restrict__ coeff,
                                                 double2* __restrict__ hsum, const int* __restrict__ skip,
                                                 const int* __restrict__ jd = nullptr) {
    if (skip && *skip) return;
    if (jd && (int)blockIdx.x > *jd) return;  // blocks beyond this step's vectors
    __shared__ double2 sh[RB / 32];
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < RG; b += RB) {
        const double2 v = partial[(int64_t)blockIdx.x * RG + b];
        acc.x += v.x;
        acc.y += v.y;
    }
    const double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) {
        coeff[blockIdx.x] = to_df4(s);
        hsum[blockIdx.x].x += s.x;
        hsum[blockIdx.x].y += s.y;
    }
}

// Whether the second Gram-Schmidt pass is needed (a test in the manner of Daniel, Gragg, Kaufman
// and Stewart): after the first pass |w'|^2 = |w|^2 - sum |h_i|^2 (Pythagoras, FP64).  One
// classical pass leaves w' orthogonal to the basis up to about u |w| / |w'|, u the working
// precision; the basis and w are double-float (u ~ 1e-14), so the pass is repeated only when
// |w'| < kReorthEta |w| (1e-4: orthogonality stays below about 1e-10, far under any GMRES
// tolerance), else *skip = 1.  wpart: the RG partials of |w|^2 before the pass.
constexpr double kReorthEta = 1e-4;
__global__ void __launch_bounds__(RB) k_reorth_decide(const double2* __restrict__ partial, const double2* __restrict__ h,
                                                      int nvec, int* __restrict__ skip,
                                                      const int* __restrict__ jd = nullptr) {
    if (jd) nvec = *jd + 1;
    const double2* wpart = partial + (size_t)nvec * RG;
    __shared__ double2 sh[RB / 32];
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < RG; b += RB) acc.x += wpart[b].x;
    for (int i = threadIdx.x; i < nvec; i += RB) acc.y += h[i].x * h[i].x + h[i].y * h[i].y;
    const double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) *skip = (s.x - s.y >= kReorthEta * kReorthEta * s.x) ? 1 : 0;
}

// one block: nrm = sqrt(sum of the RG partials of |w|^2); hsum[j1] = nrm (when j1 >= 0);
// scale = 1 / nrm as (hi, lo) (0 when nrm = 0); out[0] = nrm
__global__ void __launch_bounds__(RB) k_norm_finish(const double2* __restrict__ partial, int j1,
                                                    double2* __restrict__ hsum, float2* __restrict__ scale,
                                                    double* __restrict__ out, const int* __restrict__ jd = nullptr) {
    if (jd) j1 = *jd + 1;
    __shared__ double2 sh[RB / 32];
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < RG; b += RB) acc.x += partial[b].x;
    const double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) {
        const double n = sqrt(s.x);
        if (j1 >= 0) hsum[j1] = make_double2(n, 0.0);
        const double inv = n > 0.0 ? 1.0 / n : 0.0;
        const float ih = (float)inv;
        *scale = make_float2(ih, (float)(inv - (double)ih));
        out[0] = n;
    }
}

// b = s a with s = (hi, lo) read from device memory; with jd, b is basis vector *jd + 1 of b
__global__ void k_scale_df_dev(int64_t N, const float4* __restrict__ a, const float2* __restrict__ s,
                               float4* __restrict__ b, const int* __restrict__ jd = nullptr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (jd) b += (int64_t)(*jd + 1) * N;
    const float sh = s->x, sl = s->y;
    const float4 v = a[i];
    float4 o;
    {
        const float p = __fmul_rn(v.x, sh);
        const float q = __fmaf_rn(v.x, sl, __fmaf_rn(v.z, sh, __fmaf_rn(v.x, sh, -p)));
        fast_two_sum(p, q, o.x, o.z);
    }
    {
        const float p = __fmul_rn(v.y, sh);
        const float q = __fmaf_rn(v.y, sl, __fmaf_rn(v.w, sh, __fmaf_rn(v.y, sh, -p)));
        fast_two_sum(p, q, o.y, o.w);
    }
    b[i] = o;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

struct Arnoldi {     // device state of one GMRES cycle (FP64)
    double2* H;      // (m + 1) x m Hessenberg matrix, rotated, row-major
    double2* cs;     // m rotations (c, s), each acting on rows (i, i+1) as [[conj c, conj s], [-s, c]]
    double2* sn;
    double2* g;      // m + 1: rotated right-hand side, g[0] = beta at the cycle's start
    double* res;     // [0] |g[j+1]| / ||b||, [1] the new column's subdiagonal norm
};

// Column j: previous rotations, a new rotation for rows (j, j+1), g, the residual estimate.
__global__ void k_givens(int j, int m, const double2* __restrict__ hsum, Arnoldi A, double bnorm,
                         const int* __restrict__ jd = nullptr, const double* __restrict__ bnorm_d = nullptr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (jd) j = *jd;
    if (bnorm_d) bnorm = *bnorm_d;
    double2 h[2];  // rows i, i + 1 as the rotations sweep down
    h[0] = hsum[0];
    for (int i = 0; i < j; ++i) {
        const double2 hi1 = hsum[i + 1];
        const double2 t = cadd(cmul(cconj(A.cs[i]), h[0]), cmul(cconj(A.sn[i]), hi1));
        const double2 b = cadd(cmul(make_double2(-A.sn[i].x, -A.sn[i].y), h[0]), cmul(A.cs[i], hi1));
        A.H[(size_t)i * m + j] = t;
        h[0] = b;
    }
    const double2 hj = h[0], hj1 = hsum[j + 1];
    const double den = sqrt(hj.x * hj.x + hj.y * hj.y + hj1.x * hj1.x + hj1.y * hj1.y);
    double2 c = make_double2(1.0, 0.0), s = make_double2(0.0, 0.0);
    if (den != 0.0) {
        c = make_double2(hj.x / den, hj.y / den);
        s = make_double2(hj1.x / den, hj1.y / den);
    }
    A.cs[j] = c;
    A.sn[j] = s;
    A.H[(size_t)j * m + j] = cadd(cmul(cconj(c), hj), cmul(cconj(s), hj1));
    const double2 gj = A.g[j];
    A.g[j + 1] = cmul(make_double2(-s.x, -s.y), gj);
    A.g[j] = cmul(cconj(c), gj);
    A.res[0] = sqrt(A.g[j + 1].x * A.g[j + 1].x + A.g[j + 1].y * A.g[j + 1].y) / bnorm;
    A.res[1] = sqrt(hj1.x * hj1.x + hj1.y * hj1.y);
}

// cycle start: g = (beta, 0, ..., 0) with beta = nrm[0]
__global__ void k_cycle_start(int m, Arnoldi A, const double* __restrict__ nrm) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) A.g[i] = make_double2(i == 0 ? nrm[0] : 0.0, 0.0);
}

// y = H[0..n)^{-1} g (upper triangular) as double-float coefficients
__global__ void k_backsolve(int n, int m, Arnoldi A, double2* __restrict__ y, float4* __restrict__ coeff) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = n - 1; i >= 0; --i) {
        double2 s = A.g[i];
        for (int q = i + 1; q < n; ++q) {
            const double2 t = cmul(A.H[(size_t)i * m + q], y[q]);
            s.x -= t.x;
            s.y -= t.y;
        }
        const double2 d = A.H[(size_t)i * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd);
        coeff[i] = to_df4(y[i]);
    }
}

// sig[i] = wscale[i] (high part of basis vector *jd at user point perm[i]): the density of the
// step's matvec, read from the basis without a host-side pointer
__global__ void k_prep_basis(int64_t N, const int32_t* __restrict__ perm, const float* __restrict__ wscale,
                             const float4* __restrict__ V, const int* __restrict__ jd, float2* __restrict__ sig) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 v = V[(int64_t)(*jd) * N + perm[i]];
    const float w = wscale[i];
    sig[i] = make_float2(w * v.x, w * v.y);
}

// End of an Arnoldi step: one more iteration and one more basis vector; the cycle goes on while
// the residual estimate is above tol, the new column is non-zero, the cycle has room and the
// iteration budget is not spent.  With a graph, the decision is the while node's condition.
__global__ void k_step_end(const double* __restrict__ res, int* __restrict__ jd, int* __restrict__ itd, int m,
                           int maxit, double tol, int* __restrict__ cont, cudaGraphConditionalHandle h, int use_h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = *jd + 1, it = *itd + 1;
    *jd = j;
    *itd = it;
    const int go = (res[0] > tol && res[1] != 0.0 && j < m && it < maxit) ? 1 : 0;
    *cont = go;
    if (use_h) cudaGraphSetConditional(h, (unsigned)go);
}

// cudaGraphSetConditional(h, *act): opens (1) or closes (0) a group member's while loop
__global__ void k_cond_init(cudaGraphConditionalHandle h, const int* __restrict__ act) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, *act ? 1u : 0u);
}

namespace {

// One single right-hand-side GMRES(m) solve on a plan (Sec. 5.1's solver): its workspace, the
// pieces of a restart cycle, and what the host keeps between cycles.
struct Solver {
    hfmm_plan* P = nullptr;
    int64_t N = 0;
    int m = 0, maxit = 0;
    double tol = 0.0;
    unsigned nb = 0;
    float4* V = nullptr;
    double2 *partial = nullptr, *hsum = nullptr, *y = nullptr;
    float4* coeff = nullptr;
    Arnoldi A{};
    double* nrm = nullptr;
    float2* scale = nullptr;
    int *skip2 = nullptr, *jd = nullptr, *itd = nullptr, *contd = nullptr, *actd = nullptr;
    double* bnd = nullptr;
    double bnorm = 0.0, beta = 0.0;
    int it = 0;
    bool converged = false, done = false;
    int64_t step_launches = 0;  // kernels of one captured step

    void count(int n = 1) { P->launches += n; }

    // workspace (doubles): partials RG (m + 2) complex, hsum m + 2, H (m + 1) m, cs m, sn m,
    // g m + 1, y m (complex each), coefficients m + 2 (double-float complex), then 8 scalars:
    // residual pair, norm, scale, second-pass flag, step and iteration counters, step
    // decision and group gate, ||b||
    void init(hfmm_plan* plan) {
        P = plan;
        N = P->N;
        m = P->cfg.restart;
        tol = P->cfg.tol;
        maxit = P->cfg.max_iter;
        nb = (unsigned)((N + 255) / 256);
        const size_t n_part = 2 * (size_t)RG * (m + 2), n_hsum = 2 * (size_t)(m + 2), n_H = 2 * (size_t)(m + 1) * m,
                     n_cs = 2 * (size_t)m, n_g = 2 * (size_t)(m + 1), n_y = 2 * (size_t)m, n_coef = 2 * (size_t)(m + 2);
        const size_t n_ws = n_part + n_hsum + n_H + 2 * n_cs + n_g + n_y + n_coef + 8;
        if (P->kry_m != m) {
            if (P->gm_exec) {  // the captured step refers to the old workspace
                cudaGraphExecDestroy(P->gm_exec);
                P->gm_exec = nullptr;
            }
            P->kry.alloc((size_t)(m + 1) * N, nullptr);
            P->gw.alloc(N, nullptr);
            P->gx.alloc(N, nullptr);
            P->gb.alloc(N, nullptr);
            P->gred.alloc(n_ws, nullptr);
            P->kry_m = m;
        }
        double* ws = P->gred.p;
        partial = (double2*)ws;
        hsum = (double2*)(ws + n_part);
        A.H = (double2*)(ws + n_part + n_hsum);
        A.cs = (double2*)(ws + n_part + n_hsum + n_H);
        A.sn = A.cs + m;
        A.g = (double2*)(ws + n_part + n_hsum + n_H + 2 * n_cs);
        y = (double2*)(ws + n_part + n_hsum + n_H + 2 * n_cs + n_g);
        coeff = (float4*)(ws + n_part + n_hsum + n_H + 2 * n_cs + n_g + n_y);
        double* tail = ws + n_part + n_hsum + n_H + 2 * n_cs + n_g + n_y + n_coef;
        A.res = tail;  // 2 doubles
        nrm = tail + 2;
        scale = (float2*)(tail + 3);
        skip2 = (int*)(tail + 4);  // second Gram-Schmidt pass not needed
        jd = (int*)(tail + 5);     // step of the cycle, held on the device
        itd = jd + 1;              // iterations of the solve
        contd = (int*)(tail + 6);  // the step's decision (host-driven steps)
        actd = contd + 1;          // the solve still runs (group launches)
        bnd = tail + 7;            // ||b||
        V = P->kry.p;
    }
    void matvec(const float4* in, float4* out, cudaStream_t st) {
        launch_density_prep(P, in, VecKind::DoubleFloat, P->sig.p, st);
        run_matvec_sorted(P, 7, st);
        launch_output(P, P->phi.p, out, VecKind::DoubleFloat, st);
    }
    double norm(const float4* w, cudaStream_t st) {
        k_norm2_df<<<RG, RB, 0, st>>>(N, w, partial);
        k_reduce<<<1, RB, 0, st>>>(partial, hsum + m + 1);
        count(2);
        double2 h;
        HFMM_CUDA(cudaMemcpyAsync(&h, hsum + m + 1, sizeof(double2), cudaMemcpyDeviceToHost, st));
        host_wait(P, st);
        return std::sqrt(h.x);
    }
    void launch_norm(const float4* w, int j1, cudaStream_t st) {  // nrm, scale = 1 / nrm, hsum[j1] = nrm
        k_norm2_df<<<RG, RB, 0, st>>>(N, w, partial);
        k_norm_finish<<<1, RB, 0, st>>>(partial, j1, hsum, scale, nrm);
        count(2);
    }
    // One Arnoldi step with the step index j held on the device (stream s): the matvec of basis
    // vector j, Gram-Schmidt against the j + 1 vectors (the second pass only when the first
    // cancelled), the new basis vector, the rotations and the residual estimate, then the
    // decision to go on (the while node's condition h when use_h).  Grids are sized for the
    // cycle's longest step, so the same launches serve every j.
    void step(cudaStream_t s, cudaGraphConditionalHandle h, int use_h) {
        float4* w = P->gw.p;
        const unsigned gy = (unsigned)((m + kDotVecs - 1) / kDotVecs);
        k_prep_basis<<<nb, 256, 0, s>>>(N, P->perm.p, P->wscale.p, V, jd, P->sig.p);
        run_matvec_sorted(P, 15, s);  // every stage launched directly (a replay cannot sit in this capture)
        launch_output(P, P->phi.p, w, VecKind::DoubleFloat, s);
        HFMM_CUDA(cudaMemsetAsync(hsum, 0, sizeof(double2) * (m + 1), s));
        for (int pass = 0; pass < 2; ++pass) {
            const bool first = pass == 0;
            k_dots_df<<<dim3(RG, gy), RB, 0, s>>>(N, V, 0, w, partial, first ? nullptr : skip2, first, jd);
            k_reduce_h<<<m, RB, 0, s>>>(partial, coeff, hsum, first ? nullptr : skip2, jd);
            if (first) k_reorth_decide<<<1, RB, 0, s>>>(partial, hsum, 0, skip2, jd);
            k_axpy_df<<<nb, 256, sizeof(float4) * m, s>>>(N, V, 0, coeff, -1.f, w, first ? nullptr : skip2, jd);
        }
        k_norm2_df<<<RG, RB, 0, s>>>(N, w, partial);
        k_norm_finish<<<1, RB, 0, s>>>(partial, 0, hsum, scale, nrm, jd);
        k_scale_df_dev<<<nb, 256, 0, s>>>(N, w, scale, V, jd);
        k_givens<<<1, 32, 0, s>>>(0, m, hsum, A, 0.0, jd, bnd);
        k_step_end<<<1, 32, 0, s>>>(A.res, jd, itd, m, maxit, tol, contd, h, use_h);
        count(13);  // prep, 7 Gram-Schmidt kernels, norm, norm finish, scale, rotations, step end
        HFMM_CUDA(cudaGetLastError());
    }
    // b, x = 0, ||b||, r0 = b; false (and done) when b = 0
    bool start(const void* rhs, cudaStream_t st) {
        k_c64_to_df<<<nb, 256, 0, st>>>(N, (const float2*)rhs, P->gb.p);
        count();
        HFMM_CUDA(cudaMemsetAsync(P->gx.p, 0, sizeof(float4) * N, st));
        bnorm = norm(P->gb.p, st);
        it = 0;
        beta = bnorm;
        if (bnorm == 0.0) {
            converged = done = true;
            return false;
        }
        HFMM_CUDA(cudaMemcpyAsync(bnd, &bnorm, sizeof(double), cudaMemcpyHostToDevice, st));
        HFMM_CUDA(cudaMemsetAsync(itd, 0, sizeof(int), st));
        HFMM_CUDA(cudaMemcpyAsync(P->gw.p, P->gb.p, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
        converged = done = false;
        return true;
    }
    // V_0 = r / beta, g = (beta, 0, ...), j = 0
    void cycle_begin(cudaStream_t st) {
        launch_norm(P->gw.p, -1, st);
        k_scale_df_dev<<<nb, 256, 0, st>>>(N, P->gw.p, scale, V);
        k_cycle_start<<<1, 64, 0, st>>>(m, A, nrm);
        count(2);
        HFMM_CUDA(cudaMemsetAsync(jd, 0, sizeof(int), st));
    }
    void host_steps(cudaStream_t st) {
        for (;;) {
            step(st, cudaGraphConditionalHandle{}, 0);
            int go = 0;
            HFMM_CUDA(cudaMemcpyAsync(&go, contd, sizeof(int), cudaMemcpyDeviceToHost, st));
            host_wait(P, st);
            if (!go) break;
        }
    }
    // after the cycle's steps: y = H^{-1} g, x += V y, the true residual and its norm
    void cycle_end(cudaStream_t st, bool graph) {
        int ji[2];
        HFMM_CUDA(cudaMemcpyAsync(ji, jd, sizeof(ji), cudaMemcpyDeviceToHost, st));
        host_wait(P, st);
        const int jdone = ji[0];
        if (graph) P->launches += (int64_t)jdone * step_launches;
        it = ji[1];
        k_backsolve<<<1, 32, 0, st>>>(jdone, m, A, y, coeff);
        k_axpy_df<<<nb, 256, sizeof(float4) * jdone, st>>>(N, V, jdone, coeff, 1.f, P->gx.p);
        count(2);
        matvec(P->gx.p, P->gw.p, st);
        k_sub_df<<<nb, 256, 0, st>>>(N, P->gb.p, P->gw.p, P->gw.p);
        count();
        beta = norm(P->gw.p, st);
        converged = beta / bnorm <= tol;
        done = converged || it >= maxit;
    }
    void finish(void* x_out, cudaStream_t st) {
        k_df_to_c64<<<nb, 256, 0, st>>>(N, P->gx.p, (float2*)x_out);
        count();
        HFMM_CUDA(cudaGetLastError());
        host_wait(P, st);
    }
};

// Adds to graph g, for each solver, a while node whose body is one step of that solver
// (captured on the solver plan's own capture stream).  gated: the loop is opened or closed at
// each launch by a kernel node before it that copies the solver's device flag into the
// condition; else the condition starts at 1 at every launch.  False if any part fails.
bool add_step_loops(cudaGraph_t g, Solver* const* S, int n, bool gated) {
    for (int i = 0; i < n; ++i) {
        Solver& s = *S[i];
        MatvecGraph& MG = s.P->mvg;
        if (!MG.cap && cudaStreamCreateWithFlags(&MG.cap, cudaStreamNonBlocking) != cudaSuccess) return false;
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, gated ? 0u : 1u, gated ? 0u : cudaGraphCondAssignDefault) !=
            cudaSuccess)
            return false;
        cudaGraphNode_t gate = nullptr;
        if (gated) {
            int* act = s.actd;
            void* args[] = {&h, &act};
            cudaKernelNodeParams kp = {};
            kp.func = (void*)k_cond_init;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = args;
            if (cudaGraphAddKernelNode(&gate, g, nullptr, 0, &kp) != cudaSuccess) return false;
        }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, g, gate ? &gate : nullptr, nullptr, gate ? 1 : 0, &cp) != cudaSuccess) return false;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const int64_t l0 = s.P->launches;
        if (cudaStreamBeginCaptureToGraph(MG.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
            return false;
        bool ok = true;
        try {
            s.step(MG.cap, h, 1);
        } catch (const HfmmError&) {
            ok = false;
        }
        cudaGraph_t out = nullptr;
        ok = (cudaStreamEndCapture(MG.cap, &out) == cudaSuccess) && ok;
        s.step_launches = s.P->launches - l0;
        s.P->launches = l0;
        if (!ok) return false;
    }
    return true;
}

// a graph over the solvers' step loops, instantiated; nullptr (errors cleared) if it cannot be built
cudaGraphExec_t build_loops(Solver* const* S, int n, bool gated) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaGraphExec_t ex = nullptr;
    if (!add_step_loops(g, S, n, gated) || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    cudaGraphDestroy(g);
    cudaGetLastError();  // a capture another thread invalidated, or an unsupported node: steps from the host
    return ex;
}

}  // namespace

int run_gmres(hfmm_plan* P, const void* rhs, void* x_out, int* iters, double* relres, cudaStream_t st) {
    Solver S;
    S.init(P);
    if (!S.start(rhs, st)) {
        S.finish(x_out, st);
        *iters = 0;
        *relres = 0.0;
        return HFMM_OK;
    }
    // The whole cycle as one graph launch: a while node whose body is one step, looping on the
    // device until the step's last kernel clears its condition (no host round trip per
    // iteration).  Built once per plan and restart length; on an adaptive tree, or if building
    // fails, the host drives the same steps.
    if (!P->adaptive && !P->gm_exec) {
        Solver* one = &S;
        P->gm_exec = build_loops(&one, 1, false);
        P->gm_launches = S.step_launches;
    }
    S.step_launches = P->gm_launches;
    const bool graph = P->gm_exec != nullptr;
    P->gm_used = graph ? 1 : 0;
    while (!S.done) {
        S.cycle_begin(st);
        if (graph) HFMM_CUDA(cudaGraphLaunch(P->gm_exec, st));
        else S.host_steps(st);
        S.cycle_end(st, graph);
    }
    S.finish(x_out, st);
    *iters = S.it;
    *relres = S.beta / S.bnorm;
    return S.converged ? HFMM_OK : HFMM_NOT_CONVERGED;
}

// G independent solves (different plans, one right-hand side each) in lockstep over restart
// cycles: each cycle of every unfinished solve runs inside one shared graph launch, one gated
// while node per solve (a finished solve's loop is closed by its gate), so the requests' steps
// share a launch and proceed side by side on the device; the cycle ends run per solve.
int run_gmres_group(hfmm_plan* const* plans, int G, const void* const* rhs, void* const* x_out, int* iters,
                    double* relres, cudaStream_t st) {
    std::vector<Solver> S((size_t)G);
    std::vector<Solver*> ptr((size_t)G);
    bool adaptive = false;
    for (int g = 0; g < G; ++g) {
        S[(size_t)g].init(plans[g]);
        ptr[(size_t)g] = &S[(size_t)g];
        adaptive |= plans[g]->adaptive;
        S[(size_t)g].start(rhs[g], st);
    }
    cudaGraphExec_t ex = adaptive ? nullptr : build_loops(ptr.data(), G, true);
    struct Guard {
        cudaGraphExec_t e;
        ~Guard() {
            if (e) cudaGraphExecDestroy(e);
        }
    } guard{ex};
    for (;;) {
        bool any = false;
        for (int g = 0; g < G; ++g) any |= !S[(size_t)g].done;
        if (!any) break;
        for (int g = 0; g < G; ++g) {
            Solver& s = S[(size_t)g];
            const int act = s.done ? 0 : 1;
            HFMM_CUDA(cudaMemcpyAsync(s.actd, &act, sizeof(int), cudaMemcpyHostToDevice, st));
            if (!s.done) s.cycle_begin(st);
        }
        if (ex) {
            HFMM_CUDA(cudaGraphLaunch(ex, st));
        } else {
            for (int g = 0; g < G; ++g)
                if (!S[(size_t)g].done) S[(size_t)g].host_steps(st);
        }
        for (int g = 0; g < G; ++g)
            if (!S[(size_t)g].done) S[(size_t)g].cycle_end(st, ex != nullptr);
    }
    bool all = true;
    for (int g = 0; g < G; ++g) {
        Solver& s = S[(size_t)g];
        s.finish(x_out[g], st);
        if (iters) iters[g] = s.it;
        if (relres) relres[g] = s.bnorm > 0.0 ? s.beta / s.bnorm : 0.0;
        all &= s.converged;
        s.P->gm_used = ex ? 1 : 0;
    }
    return all ? HFMM_OK : HFMM_NOT_CONVERGED;
}

// ============================================================== R systems in lockstep
// Vectors hold R right-hand sides, [r][N] double-float; kernels take the right-hand side
// from blockIdx.y (or .z) and otherwise do what their single right-hand-side versions do.

// partial[(r * nvec + i) * RG + blk] = sum over the block's rows of conj(V_i[r]) w[r]
__global__ void __launch_bounds__(RB) k_dots_bdf(int64_t N, int R, const float4* __restrict__ V, int nvec,
                                                 const float4* __restrict__ w, double2* __restrict__ partial) {
    __shared__ double2 sh[RB / 32];
    const int r = blockIdx.z, i0 = blockIdx.y * kDotVecs;
    const int nv = min(kDotVecs, nvec - i0);
    const float4* wr = w + (int64_t)r * N;
    Acc re[kDotVecs], im[kDotVecs];
    for (int64_t n = (int64_t)blockIdx.x * RB + threadIdx.x; n < N; n += (int64_t)RG * RB) {
        const float4 b = wr[n];
        float4 av[kDotVecs];  // all the row's loads in flight first (absent vectors: zero)
#pragma unroll
        for (int c = 0; c < kDotVecs; ++c)
            av[c] = c < nv ? V[((int64_t)(i0 + c) * R + r) * N + n] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kDotVecs; ++c) {
            const float4 a = av[c];
            re[c].add_prod(a.x, a.z, b.x, b.z);
            re[c].add_prod(a.y, a.w, b.y, b.w);
            im[c].add_prod(a.x, a.z, b.y, b.w);
            im[c].add_prod(-a.y, -a.w, b.x, b.z);
        }
    }
#pragma unroll
    for (int c = 0; c < kDotVecs; ++c) {
        if (c >= nv) break;
        const double2 s = block_sum2(make_double2(re[c].value(), im[c].value()), sh);
        if (threadIdx.x == 0) partial[((int64_t)r * nvec + i0 + c) * RG + blockIdx.x] = s;
    }
}

// partial[r * RG + blk] = sum |w[r]|^2 over the block's rows
__global__ void __launch_bounds__(RB) k_norm2_bdf(int64_t N, const float4* __restrict__ w,
                                                  double2* __restrict__ partial) {
    __shared__ double2 sh[RB / 32];
    const float4* wr = w + (int64_t)blockIdx.y * N;
    Acc a;
    for (int64_t n = (int64_t)blockIdx.x * RB + threadIdx.x; n < N; n += (int64_t)RG * RB) {
        const float4 b = wr[n];
        a.add_prod(b.x, b.z, b.x, b.z);
        a.add_prod(b.y, b.w, b.y, b.w);
    }
    const double2 s = block_sum2(make_double2(a.value(), 0.0), sh);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * RG + blockIdx.x] = s;
}

// x[r] += sign * sum_i c[r][i] V_i[r]   (c: double-float complex, [R][nvec])
__global__ void k_axpy_bdf(int64_t N, int R, const float4* __restrict__ V, int nvec, const float4* __restrict__ cdf,
                           float sign, float4* __restrict__ x) {
    extern __shared__ float4 hs[];
    const int r = blockIdx.y;
    for (int q = threadIdx.x; q < nvec; q += blockDim.x) hs[q] = cdf[(int64_t)r * nvec + q];
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    Acc ar, ai;
    for (int i = 0; i < nvec; ++i) {
        const float4 a = V[((int64_t)i * R + r) * N + n], h = hs[i];
        ar.add_prod(h.x, h.z, a.x, a.z);
        ar.add_prod(-h.y, -h.w, a.y, a.w);
        ai.add_prod(h.x, h.z, a.y, a.w);
        ai.add_prod(h.y, h.w, a.x, a.z);
    }
    float4* xr = x + (int64_t)r * N;
    float4 o = xr[n];
    float sh, sl;
    two_sum(ar.s, ar.c, sh, sl);
    df_add(o.x, o.z, sign * sh, sign * sl, o.x, o.z);
    two_sum(ai.s, ai.c, sh, sl);
    df_add(o.y, o.w, sign * sh, sign * sl, o.y, o.w);
    xr[n] = o;
}

// b[r] = s_r a[r], s_r = scale[r].x + scale[r].y
__global__ void k_scale_bdf(int64_t N, const float4* __restrict__ a, const float2* __restrict__ scale,
                            float4* __restrict__ b) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.y;
    const float sh = scale[r].x, sl = scale[r].y;
    const float4 v = a[(int64_t)r * N + n];
    float4 o;
    {
        const float p = __fmul_rn(v.x, sh);
        const float q = __fmaf_rn(v.x, sl, __fmaf_rn(v.z, sh, __fmaf_rn(v.x, sh, -p)));
        fast_two_sum(p, q, o.x, o.z);
    }
    {
        const float p = __fmul_rn(v.y, sh);
        const float q = __fmaf_rn(v.y, sl, __fmaf_rn(v.w, sh, __fmaf_rn(v.y, sh, -p)));
        fast_two_sum(p, q, o.y, o.w);
    }
    b[(int64_t)r * N + n] = o;
}

namespace {
struct BCtx {
    hfmm_plan* P;
    cudaStream_t st;
    int64_t N;
    int R;
    unsigned nb;
    double2* partial;  // RG * R * (m + 2)
    double2* small;    // R * (m + 2)
    float4* coeff;     // R * (m + 2) double-float coefficients
    float2* scales;    // R double-float scale factors

    void count(int n = 1) { P->launches += n; }
    int64_t RN() const { return (int64_t)R * N; }
    unsigned nbRN() const { return (unsigned)((RN() + 255) / 256); }
    void matvec(const float4* in, float4* out) {
        k_df_to_c64<<<nbRN(), 256, 0, st>>>(RN(), in, P->bin.p);
        batched_matvec(P, P->bin.p, P->bout.p, R, st);
        k_c64_to_df<<<nbRN(), 256, 0, st>>>(RN(), P->bout.p, out);
        count(2);
    }
    std::vector<double> norms(const float4* w) {
        k_norm2_bdf<<<dim3(RG, R), RB, 0, st>>>(N, w, partial);
        k_reduce<<<R, RB, 0, st>>>(partial, small);
        count(2);
        std::vector<double2> h(R);
        HFMM_CUDA(cudaMemcpyAsync(h.data(), small, sizeof(double2) * R, cudaMemcpyDeviceToHost, st));
        host_wait(P, st);
        std::vector<double> out(R);
        for (int r = 0; r < R; ++r) out[r] = std::sqrt(h[r].x);
        return out;
    }
    // b[r] = s[r] a[r] (s on the host, FP64)
    void scale(const float4* a, const std::vector<double>& s, float4* b) {
        std::vector<float2> sf(R);
        for (int r = 0; r < R; ++r) split_df(s[r], sf[r].x, sf[r].y);
        HFMM_CUDA(cudaMemcpyAsync(scales, sf.data(), sizeof(float2) * R, cudaMemcpyHostToDevice, st));
        k_scale_bdf<<<dim3(nb, R), 256, 0, st>>>(N, a, scales, b);
        count();
    }
    // x[r] += sign * V[0..nvec)[r] c[r]
    void axpy(const float4* V, int nvec, const std::vector<std::vector<cd>>& c, float sign, float4* x) {
        std::vector<float4> cf((size_t)R * nvec);
        for (int r = 0; r < R; ++r)
            for (int i = 0; i < nvec; ++i) {
                float rh, rl, ih, il;
                const cd v = i < (int)c[r].size() ? c[r][i] : cd(0);
                split_df(v.real(), rh, rl);
                split_df(v.imag(), ih, il);
                cf[(size_t)r * nvec + i] = make_float4(rh, ih, rl, il);
            }
        HFMM_CUDA(cudaMemcpyAsync(coeff, cf.data(), sizeof(float4) * cf.size(), cudaMemcpyHostToDevice, st));
        k_axpy_bdf<<<dim3(nb, R), 256, sizeof(float4) * nvec, st>>>(N, R, V, nvec, coeff, sign, x);
        count();
    }
    // h[r] = V[0..nvec)[r]^H w[r], then w[r] -= V[r] h[r]; adds into hsum
    void cgs_pass(const float4* V, int nvec, float4* w, std::vector<std::vector<cd>>& hsum) {
        k_dots_bdf<<<dim3(RG, (nvec + kDotVecs - 1) / kDotVecs, R), RB, 0, st>>>(N, R, V, nvec, w, partial);
        k_reduce<<<R * nvec, RB, 0, st>>>(partial, small);
        count(2);
        std::vector<double2> h((size_t)R * nvec);
        HFMM_CUDA(cudaMemcpyAsync(h.data(), small, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
        host_wait(P, st);
        std::vector<std::vector<cd>> hc(R, std::vector<cd>(nvec));
        for (int r = 0; r < R; ++r)
            for (int i = 0; i < nvec; ++i) {
                hc[r][i] = cd(h[(size_t)r * nvec + i].x, h[(size_t)r * nvec + i].y);
                hsum[r][i] += hc[r][i];
            }
        axpy(V, nvec, hc, -1.f, w);
    }
};
}  // namespace

int run_gmres_batched(hfmm_plan* P, const float2* rhs, float2* x_out, int R, int* iters, double* relres,
                      cudaStream_t st) {
    const int64_t N = P->N;
    const int m = P->cfg.restart;
    const double tol = P->cfg.tol;
    const int maxit = P->cfg.max_iter;
    const int64_t RN = (int64_t)R * N;
    if (P->bkry_m != m || P->bkry_R != R) {
        P->bkry.alloc((size_t)(m + 1) * RN, nullptr);
        P->bgw.alloc(RN, nullptr);
        P->bgx.alloc(RN, nullptr);
        P->bgb.alloc(RN, nullptr);
        P->bin.alloc(RN, nullptr);
        P->bout.alloc(RN, nullptr);
        P->bred.alloc((size_t)2 * RG * R * (m + 2) + 2 * (size_t)R * (m + 2) + 2 * (size_t)R * (m + 2) + 2 * R,
                      nullptr);
        P->bkry_m = m;
        P->bkry_R = R;
    }
    double2* red = (double2*)P->bred.p;
    double2* small = red + (size_t)RG * R * (m + 2);
    float4* coeff = reinterpret_cast<float4*>(small + (size_t)R * (m + 2));
    float2* scales = reinterpret_cast<float2*>(coeff + (size_t)R * (m + 2));
    BCtx c{P, st, N, R, (unsigned)((N + 255) / 256), red, small, coeff, scales};
    float4* V = P->bkry.p;
    float4 *w = P->bgw.p, *xg = P->bgx.p, *bg = P->bgb.p;
    k_c64_to_df<<<c.nbRN(), 256, 0, st>>>(RN, rhs, bg);
    c.count();
    HFMM_CUDA(cudaMemsetAsync(xg, 0, sizeof(float4) * RN, st));
    const std::vector<double> bnorm = c.norms(bg);
    std::vector<double> beta = bnorm;
    std::vector<char> done(R, 0);  // converged (or zero right-hand side)
    for (int r = 0; r < R; ++r) {
        iters[r] = 0;
        relres[r] = 0.0;
        if (bnorm[r] == 0.0) done[r] = 1;
    }
    HFMM_CUDA(cudaMemcpyAsync(w, bg, sizeof(float4) * RN, cudaMemcpyDeviceToDevice, st));
    int it = 0;
    auto all_done = [&]() {
        for (int r = 0; r < R; ++r)
            if (!done[r]) return false;
        return true;
    };
    while (it < maxit && !all_done()) {
        // V_0[r] = r0 / beta (zero for the finished right-hand sides, which then stay inert)
        std::vector<double> s0(R);
        for (int r = 0; r < R; ++r) s0[r] = done[r] ? 0.0 : 1.0 / beta[r];
        c.scale(w, s0, V);
        std::vector<std::vector<cd>> H(R, std::vector<cd>((size_t)(m + 1) * m, cd(0))), cs(R, std::vector<cd>(m)),
            sn(R, std::vector<cd>(m)), g(R, std::vector<cd>(m + 1, cd(0)));
        std::vector<int> jdone(R, 0);
        std::vector<char> active(R);
        for (int r = 0; r < R; ++r) {
            g[r][0] = done[r] ? 0.0 : beta[r];
            active[r] = !done[r];
        }
        for (int j = 0; j < m && it < maxit; ++j) {
            c.matvec(V + (int64_t)j * RN, w);
            std::vector<std::vector<cd>> h(R, std::vector<cd>(j + 2, cd(0)));
            c.cgs_pass(V, j + 1, w, h);
            c.cgs_pass(V, j + 1, w, h);
            const std::vector<double> hn = c.norms(w);
            std::vector<double> sc(R);
            for (int r = 0; r < R; ++r) sc[r] = (active[r] && hn[r] > 0.0) ? 1.0 / hn[r] : 0.0;
            c.scale(w, sc, V + (int64_t)(j + 1) * RN);
            ++it;
            bool any = false;
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                auto& hr = h[r];
                hr[j + 1] = hn[r];
                for (int i = 0; i < j; ++i) {
                    const cd t = std::conj(cs[r][i]) * hr[i] + std::conj(sn[r][i]) * hr[i + 1];
                    hr[i + 1] = -sn[r][i] * hr[i] + cs[r][i] * hr[i + 1];
                    hr[i] = t;
                }
                const double den = std::sqrt(std::norm(hr[j]) + std::norm(hr[j + 1]));
                if (den == 0.0) {
                    cs[r][j] = 1.0;
                    sn[r][j] = 0.0;
                } else {
                    cs[r][j] = hr[j] / den;
                    sn[r][j] = hr[j + 1] / den;
                }
                hr[j] = std::conj(cs[r][j]) * hr[j] + std::conj(sn[r][j]) * hr[j + 1];
                hr[j + 1] = 0.0;
                g[r][j + 1] = -sn[r][j] * g[r][j];
                g[r][j] = std::conj(cs[r][j]) * g[r][j];
                for (int i = 0; i <= j; ++i) H[r][(size_t)i * m + j] = hr[i];
                jdone[r] = j + 1;
                iters[r] = it;
                if (std::abs(g[r][j + 1]) / bnorm[r] <= tol || hn[r] == 0.0) active[r] = 0;  // stop its process
                any = any || active[r];
            }
            if (!any) break;
        }
        // y_r = H_r^{-1} g_r (FP64), x[r] += V[r] y_r
        std::vector<std::vector<cd>> y(R);
        int jmax = 0;
        for (int r = 0; r < R; ++r) {
            const int jd = done[r] ? 0 : jdone[r];
            y[r].assign(jd, cd(0));
            for (int i = jd - 1; i >= 0; --i) {
                cd s = g[r][i];
                for (int q = i + 1; q < jd; ++q) s -= H[r][(size_t)i * m + q] * y[r][q];
                y[r][i] = s / H[r][(size_t)i * m + i];
            }
            jmax = std::max(jmax, jd);
        }
        if (jmax > 0) c.axpy(V, jmax, y, 1.f, xg);
        // true residuals r = b - A x
        c.matvec(xg, w);
        k_sub_df<<<c.nbRN(), 256, 0, st>>>(RN, bg, w, w);
        c.count();
        beta = c.norms(w);
        for (int r = 0; r < R; ++r) {
            if (bnorm[r] == 0.0) continue;
            relres[r] = beta[r] / bnorm[r];
            if (relres[r] <= tol) done[r] = 1;
        }
    }
    k_df_to_c64<<<c.nbRN(), 256, 0, st>>>(RN, xg, x_out);
    c.count();
    HFMM_CUDA(cudaGetLastError());
    host_wait(P, st);
    return all_done() ? HFMM_OK : HFMM_NOT_CONVERGED;
}

// ============================================================== mixed-precision refinement
// x += d (complex64 correction into a double-float iterate)
__global__ void k_add_c64_to_df(int64_t N, const float2* __restrict__ d, float4* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 o = x[i];
    const float2 v = d[i];
    df_add(o.x, o.z, v.x, 0.f, o.x, o.z);
    df_add(o.y, o.w, v.y, 0.f, o.y, o.w);
    x[i] = o;
}

int run_refinement(hfmm_plan* Pi, hfmm_plan* Po, const float2* rhs, float2* x_out, double tol, int max_outer,
                   int* outer_iters, int* inner_iters, double* relres, cudaStream_t st) {
    const int64_t N = Pi->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (!Pi->rb.p || Pi->rb.n != (size_t)N) {
        Pi->rb.alloc(N, nullptr);
        Pi->rx.alloc(N, nullptr);
        Pi->rr.alloc(N, nullptr);
        Pi->r32.alloc(N, nullptr);
        Pi->d32.alloc(N, nullptr);
        Pi->rred.alloc((size_t)2 * RG + 2, nullptr);
    }
    double2* partial = (double2*)Pi->rred.p;
    double2* small = partial + RG;
    auto norm = [&](const float4* w) {
        k_norm2_df<<<RG, RB, 0, st>>>(N, w, partial);
        k_reduce<<<1, RB, 0, st>>>(partial, small);
        Pi->launches += 2;
        double2 h;
        HFMM_CUDA(cudaMemcpyAsync(&h, small, sizeof(double2), cudaMemcpyDeviceToHost, st));
        host_wait(Pi, st);
        return std::sqrt(h.x);
    };
    // A_outer applied to the iterate: on a precision = 1 plan the near field and correction in
    // FP64 on the whole double-float iterate (far field FP32); else the FP32 operator on its
    // high part
    auto outer_residual = [&]() {
        if (Po->cfg.precision == 1) {
            run_matvec_df(Po, Pi->rx.p, Pi->rr.p, 7, st);
        } else {
            launch_density_prep(Po, Pi->rx.p, VecKind::DoubleFloat, Po->sig.p, st);
            run_matvec_sorted(Po, 7, st);
            launch_output(Po, Po->phi.p, Pi->rr.p, VecKind::DoubleFloat, st);
        }
        k_sub_df<<<nb, 256, 0, st>>>(N, Pi->rb.p, Pi->rr.p, Pi->rr.p);
        Pi->launches += 1;
        return norm(Pi->rr.p);
    };
    k_c64_to_df<<<nb, 256, 0, st>>>(N, rhs, Pi->rb.p);
    HFMM_CUDA(cudaMemsetAsync(Pi->rx.p, 0, sizeof(float4) * N, st));
    Pi->launches += 1;
    const double bnorm = norm(Pi->rb.p);
    int outer = 0, inner = 0;
    double rel = 0.0;
    if (bnorm > 0.0) {
        HFMM_CUDA(cudaMemcpyAsync(Pi->rr.p, Pi->rb.p, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
        rel = 1.0;
        while (rel > tol && outer < max_outer) {
            // inner solve on the residual (rounded to FP32), correction added in double-float
            k_df_to_c64<<<nb, 256, 0, st>>>(N, Pi->rr.p, Pi->r32.p);
            Pi->launches += 1;
            int it = 0;
            double rr_in = 0.0;
            run_gmres(Pi, Pi->r32.p, Pi->d32.p, &it, &rr_in, st);  // a stalled inner solve still helps
            inner += it;
            k_add_c64_to_df<<<nb, 256, 0, st>>>(N, Pi->d32.p, Pi->rx.p);
            Pi->launches += 1;
            ++outer;
            rel = outer_residual() / bnorm;
        }
    } else {
        HFMM_CUDA(cudaMemsetAsync(Pi->rx.p, 0, sizeof(float4) * N, st));
    }
    k_df_to_c64<<<nb, 256, 0, st>>>(N, Pi->rx.p, x_out);
    Pi->launches += 1;
    HFMM_CUDA(cudaGetLastError());
    host_wait(Pi, st);
    if (outer_iters) *outer_iters = outer;
    if (inner_iters) *inner_iters = inner;
    if (relres) *relres = rel;
    return rel <= tol ? HFMM_OK : HFMM_NOT_CONVERGED;
}

}  // namespace hfmm
