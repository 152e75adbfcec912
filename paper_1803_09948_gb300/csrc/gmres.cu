// Restarted GMRES(m) on the device (the paper's solver: GMRES with the FMM as
// the matvec, exit at a relative residual of 1e-4; Sec. 1, 5.1, 6.4).
//
// Krylov basis, Gram-Schmidt (two classical passes), norms and the solution
// update run in FP64 on the GPU; the matvec is the FP32 FMM.  The (m+1) x m
// Hessenberg matrix and its Givens rotations live on the host: one small
// device-to-host copy per iteration.
#include <cmath>
#include <complex>
#include <vector>

#include "hfmm_internal.cuh"

namespace hfmm {

using cd = std::complex<double>;

static constexpr int RB = 256;  // threads per reduction block
static constexpr int RG = 296;  // reduction blocks per vector (2 per SM)

__global__ void k_f2d(int64_t N, const float2* __restrict__ a, double2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_double2(a[i].x, a[i].y);
}
__global__ void k_d2f(int64_t N, const double2* __restrict__ a, float2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_scale(int64_t N, const double2* __restrict__ a, double s, double2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_double2(s * a[i].x, s * a[i].y);
}
__global__ void k_sub(int64_t N, const double2* __restrict__ a, const double2* __restrict__ b,
                      double2* __restrict__ c) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) c[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

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

// partial[i * RG + blk] = sum over the block's rows of conj(V_i) w   (grid RG x nvec)
__global__ void __launch_bounds__(RB) k_dots(int64_t N, const double2* __restrict__ V, const double2* __restrict__ w,
                                             double2* __restrict__ partial) {
    __shared__ double2 sh[RB / 32];
    int i = blockIdx.y;
    const double2* v = V + (int64_t)i * N;
    double2 acc = make_double2(0, 0);
    for (int64_t r = (int64_t)blockIdx.x * RB + threadIdx.x; r < N; r += (int64_t)RG * RB) {
        double2 a = v[r], b = w[r];
        acc.x += a.x * b.x + a.y * b.y;
        acc.y += a.x * b.y - a.y * b.x;
    }
    double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) partial[(int64_t)i * RG + blockIdx.x] = s;
}

// partial[blk] = sum |w|^2 over the block's rows
__global__ void __launch_bounds__(RB) k_norm2(int64_t N, const double2* __restrict__ w, double2* __restrict__ partial) {
    __shared__ double2 sh[RB / 32];
    double2 acc = make_double2(0, 0);
    for (int64_t r = (int64_t)blockIdx.x * RB + threadIdx.x; r < N; r += (int64_t)RG * RB) {
        double2 b = w[r];
        acc.x += b.x * b.x + b.y * b.y;
    }
    double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[i] = sum_b partial[i * RG + b]   (one block per vector)
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

// w -= sum_i h_i V_i
__global__ void k_update(int64_t N, const double2* __restrict__ V, int nvec, const double2* __restrict__ h,
                         double2* __restrict__ w) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double2 acc = w[r];
    for (int i = 0; i < nvec; ++i) {
        double2 a = V[(int64_t)i * N + r], c = h[i];
        acc.x -= c.x * a.x - c.y * a.y;
        acc.y -= c.x * a.y + c.y * a.x;
    }
    w[r] = acc;
}

// x += sum_i y_i V_i
__global__ void k_combine(int64_t N, const double2* __restrict__ V, int nvec, const double2* __restrict__ y,
                          double2* __restrict__ x) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double2 acc = x[r];
    for (int i = 0; i < nvec; ++i) {
        double2 a = V[(int64_t)i * N + r], c = y[i];
        acc.x += c.x * a.x - c.y * a.y;
        acc.y += c.x * a.y + c.y * a.x;
    }
    x[r] = acc;
}

namespace {
struct Ctx {
    hfmm_plan* P;
    cudaStream_t st;
    int64_t N;
    unsigned nb;
    double2* partial;  // RG * (m + 1)
    double2* small;    // m + 2 values

    void count(int n = 1) { P->launches += n; }
    void matvec(const double2* in, double2* out) {
        launch_density_prep(P, in, true, P->sig.p, st);
        run_matvec_sorted(P, 7, st);
        launch_output(P, P->phi.p, out, true, st);
    }
    double norm(const double2* w) {
        k_norm2<<<RG, RB, 0, st>>>(N, w, partial);
        k_reduce<<<1, RB, 0, st>>>(partial, small);
        count(2);
        double2 h;
        HFMM_CUDA(cudaMemcpyAsync(&h, small, sizeof(double2), cudaMemcpyDeviceToHost, st));
        HFMM_CUDA(cudaStreamSynchronize(st));
        return std::sqrt(h.x);
    }
    // h = V[0..nvec)^H w (device, in small), then w -= V h; adds h into hsum
    void cgs_pass(const double2* V, int nvec, double2* w, std::vector<cd>& hsum) {
        k_dots<<<dim3(RG, nvec), RB, 0, st>>>(N, V, w, partial);
        k_reduce<<<nvec, RB, 0, st>>>(partial, small);
        k_update<<<nb, 256, 0, st>>>(N, V, nvec, small, w);
        count(3);
        std::vector<double2> h(nvec);
        HFMM_CUDA(cudaMemcpyAsync(h.data(), small, sizeof(double2) * nvec, cudaMemcpyDeviceToHost, st));
        HFMM_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < nvec; ++i) hsum[i] += cd(h[i].x, h[i].y);
    }
};
}  // namespace

int run_gmres(hfmm_plan* P, const void* rhs, void* x_out, int* iters, double* relres, cudaStream_t st) {
    const int64_t N = P->N;
    const int m = P->cfg.restart;
    const double tol = P->cfg.tol;
    const int maxit = P->cfg.max_iter;
    if (P->kry_m != m) {
        P->kry.alloc((size_t)(m + 1) * N, nullptr);
        P->gw.alloc(N, nullptr);
        P->gx.alloc(N, nullptr);
        P->gb.alloc(N, nullptr);
        P->gred.alloc((size_t)2 * RG * (m + 2) + 2 * (m + 2), nullptr);
        P->kry_m = m;
    }
    Ctx c{P, st, N, (unsigned)((N + 255) / 256), (double2*)P->gred.p, (double2*)P->gred.p + (size_t)RG * (m + 2)};
    double2* V = P->kry.p;
    k_f2d<<<c.nb, 256, 0, st>>>(N, (const float2*)rhs, P->gb.p);
    c.count();
    HFMM_CUDA(cudaMemsetAsync(P->gx.p, 0, sizeof(double2) * N, st));
    double bnorm = c.norm(P->gb.p);
    if (bnorm == 0.0) {
        k_d2f<<<c.nb, 256, 0, st>>>(N, P->gx.p, (float2*)x_out);
        c.count();
        HFMM_CUDA(cudaStreamSynchronize(st));
        *iters = 0;
        *relres = 0.0;
        return HFMM_OK;
    }
    // r0 = b (x0 = 0)
    HFMM_CUDA(cudaMemcpyAsync(P->gw.p, P->gb.p, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    double beta = bnorm;
    int it = 0;
    bool converged = false;
    while (it < maxit && !converged) {
        k_scale<<<c.nb, 256, 0, st>>>(N, P->gw.p, 1.0 / beta, V);
        c.count();
        std::vector<cd> H((size_t)(m + 1) * m, cd(0)), cs(m), sn(m), g(m + 1, cd(0));
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m && it < maxit; ++j) {
            double2* w = P->gw.p;
            c.matvec(V + (int64_t)j * N, w);
            std::vector<cd> h(j + 2, cd(0));
            c.cgs_pass(V, j + 1, w, h);
            c.cgs_pass(V, j + 1, w, h);
            double hn = c.norm(w);
            h[j + 1] = hn;
            if (hn > 0.0) {
                k_scale<<<c.nb, 256, 0, st>>>(N, w, 1.0 / hn, V + (int64_t)(j + 1) * N);
                c.count();
            }
            // previous rotations, each acting on rows (i, i+1) as [[conj c, conj s], [-s, c]]
            for (int i = 0; i < j; ++i) {
                cd t = std::conj(cs[i]) * h[i] + std::conj(sn[i]) * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t;
            }
            double den = std::sqrt(std::norm(h[j]) + std::norm(h[j + 1]));
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = h[j] / den;
                sn[j] = h[j + 1] / den;
            }
            h[j] = std::conj(cs[j]) * h[j] + std::conj(sn[j]) * h[j + 1];
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = std::conj(cs[j]) * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
            ++it;
            jdone = j + 1;
            if (std::abs(g[j + 1]) / bnorm <= tol || hn == 0.0) break;
        }
        // y = H^{-1} g (upper triangular), x += V y
        std::vector<cd> y(jdone);
        for (int i = jdone - 1; i >= 0; --i) {
            cd s = g[i];
            for (int q = i + 1; q < jdone; ++q) s -= H[(size_t)i * m + q] * y[q];
            y[i] = s / H[(size_t)i * m + i];
        }
        std::vector<double2> yd(jdone);
        for (int i = 0; i < jdone; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
        HFMM_CUDA(cudaMemcpyAsync(c.small, yd.data(), sizeof(double2) * jdone, cudaMemcpyHostToDevice, st));
        k_combine<<<c.nb, 256, 0, st>>>(N, V, jdone, c.small, P->gx.p);
        c.count();
        // true residual r = b - A x
        c.matvec(P->gx.p, P->gw.p);
        k_sub<<<c.nb, 256, 0, st>>>(N, P->gb.p, P->gw.p, P->gw.p);
        c.count();
        beta = c.norm(P->gw.p);
        converged = beta / bnorm <= tol;
    }
    k_d2f<<<c.nb, 256, 0, st>>>(N, P->gx.p, (float2*)x_out);
    c.count();
    HFMM_CUDA(cudaGetLastError());
    HFMM_CUDA(cudaStreamSynchronize(st));
    *iters = it;
    *relres = beta / bnorm;
    return converged ? HFMM_OK : HFMM_NOT_CONVERGED;
}

}  // namespace hfmm
