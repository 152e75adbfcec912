// FP64 near field and correction: the accurate operator that forms the outer residual of the
// mixed-precision refinement (the GMRES solve of Sec. 5.1 / 6.4 taken to a tighter residual).
//
// The matvec is split as in the fast operator (Eq. 10 with the point rule of Eq. 7 away from the
// near sets, Sec. 2.2's corrections on them):
//     (Z s)_i = sum_{j != i, j in the near leaves of i} w_j G(x_i, x_j) s_j    (near field, P2P)
//             + far field of the same point sum (FMM, FP32 here)
//             + sum_j C_ij s_j                                                   (correction)
// On a plan created with precision = 1 the first and last terms are evaluated in FP64 from FP64
// positions, weights, quadrature nodes and correction values, on the double-float density
// (hi + lo); the far field takes the density's FP32 high part and is added in FP64.
#include <math.h>

#include "hfmm_internal.cuh"

namespace hfmm {

namespace {

constexpr double kPiD = 3.14159265358979323846;

// sorted point i: FP64 position and the scaled weight k w / (4 pi)
__global__ void k_acc_points(int64_t N, const int32_t* __restrict__ perm, const double* __restrict__ x64,
                             const double* __restrict__ w_user, double k, PointW64* __restrict__ xw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t u = perm[i];
    xw[i] = PointW64{x64[3 * u], x64[3 * u + 1], x64[3 * u + 2], k * w_user[u] / (4.0 * kPiD)};
}

// sig64[i] = (k w_i / (4 pi)) (hi + lo) of the user-order double-float density
__global__ void k_acc_prep(int64_t N, const int32_t* __restrict__ perm, const PointW64* __restrict__ xw,
                           const float4* __restrict__ in, double2* __restrict__ sig64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 v = in[perm[i]];
    const double w = xw[i].w;
    sig64[i] = make_double2(w * ((double)v.x + (double)v.z), w * ((double)v.y + (double)v.w));
}

// One block per target leaf: phi64[i] = far[i] (if given) + sum over the leaf's own points and
// its near leaves' points j != i of sig64_j exp(i k R) / (k R).
__global__ void __launch_bounds__(128) k_acc_near(const int32_t* __restrict__ leaf_start,
                                                  const int32_t* __restrict__ nbr_ptr,
                                                  const int32_t* __restrict__ nbr, const PointW64* __restrict__ xw,
                                                  const double2* __restrict__ sig64, double k,
                                                  const float2* __restrict__ far, double2* __restrict__ phi64) {
    const int b = blockIdx.x;
    const int i0 = leaf_start[b], i1 = leaf_start[b + 1];
    const int n0 = nbr_ptr[b], n1 = nbr_ptr[b + 1];
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
        const PointW64 t = xw[i];
        double ar = 0.0, ai = 0.0;
        for (int q = n0 - 1; q < n1; ++q) {  // q = n0 - 1: the leaf itself
            const int sl = q < n0 ? b : nbr[q];
            if (q >= n0 && sl == b) continue;
            const int j1 = leaf_start[sl + 1];
            for (int j = leaf_start[sl]; j < j1; ++j) {
                if (j == i) continue;
                const PointW64 s = xw[j];
                const double dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
                const double u = k * sqrt(dx * dx + dy * dy + dz * dz);
                double sn, cs;
                sincos(u, &sn, &cs);
                const double2 g = sig64[j];
                const double inv = 1.0 / u;
                ar += (g.x * cs - g.y * sn) * inv;
                ai += (g.x * sn + g.y * cs) * inv;
            }
        }
        if (far) {
            const float2 f = far[i];
            ar += (double)f.x;
            ai += (double)f.y;
        }
        phi64[i] = make_double2(ar, ai);
    }
}

__global__ void k_acc_init(int64_t N, const float2* __restrict__ far, double2* __restrict__ phi64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    phi64[i] = far ? make_double2((double)far[i].x, (double)far[i].y) : make_double2(0.0, 0.0);
}

// phi64[row] += sum_e C[e] sig64[col[e]] (one thread per row)
__global__ void k_acc_corr(int64_t N, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, const double2* __restrict__ sig64,
                           double2* __restrict__ phi64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double ar = 0.0, ai = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const double2 v = val[e], g = sig64[col[e]];
        ar += v.x * g.x - v.y * g.y;
        ai += v.x * g.y + v.y * g.x;
    }
    const double2 p = phi64[i];
    phi64[i] = make_double2(p.x + ar, p.y + ai);
}

// user-order double-float output (re_hi, im_hi, re_lo, im_lo)
__global__ void k_acc_out(int64_t N, const int32_t* __restrict__ perm, const double2* __restrict__ phi64,
                          float4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 v = phi64[i];
    const float hr = (float)v.x, hi = (float)v.y;
    out[perm[i]] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
}

}  // namespace

void accurate_setup(hfmm_plan* P, cudaStream_t st) {
    DBuf<double> w;
    w.upload(P->host_w, nullptr, st);
    P->acc_xw.alloc((size_t)P->N, &P->dev_bytes);
    P->acc_sig.alloc((size_t)P->N, &P->dev_bytes);
    P->acc_phi.alloc((size_t)P->N, &P->dev_bytes);
    k_acc_points<<<(unsigned)((P->N + 255) / 256), 256, 0, st>>>(P->N, P->perm.p, P->x64.p, w.p, P->k,
                                                                  P->acc_xw.p);
    HFMM_CUDA(cudaGetLastError());
    HFMM_CUDA(cudaStreamSynchronize(st));  // w is freed at the end of this scope
}

void run_matvec_df(hfmm_plan* P, const float4* in, float4* out, int parts, cudaStream_t st) {
    const int64_t N = P->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    k_acc_prep<<<nb, 256, 0, st>>>(N, P->perm.p, P->acc_xw.p, in, P->acc_sig.p);
    ++P->launches;
    const float2* far = nullptr;
    if (parts & 2) {  // the far field (FP32) from the density's high part
        launch_density_prep(P, in, VecKind::DoubleFloat, P->sig.p, st);
        run_matvec_sorted(P, 2, st);
        far = P->phi.p;
    }
    if (parts & 1) {
        k_acc_near<<<(unsigned)P->nleaf, 128, 0, st>>>(P->leaf_start.p, P->nbr_ptr.p, P->nbr.p, P->acc_xw.p,
                                                        P->acc_sig.p, P->k, far, P->acc_phi.p);
    } else {
        k_acc_init<<<nb, 256, 0, st>>>(N, far, P->acc_phi.p);
    }
    ++P->launches;
    if (parts & 4) {
        k_acc_corr<<<nb, 256, 0, st>>>(N, P->corr_ptr.p, P->corr_col.p, P->corr_val64.p, P->acc_sig.p,
                                        P->acc_phi.p);
        ++P->launches;
    }
    k_acc_out<<<nb, 256, 0, st>>>(N, P->perm.p, P->acc_phi.p, out);
    ++P->launches;
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
