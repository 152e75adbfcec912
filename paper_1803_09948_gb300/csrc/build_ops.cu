// Plan-time kernels: translation operators (FP64) and the sparse self/near correction
// (FP64 geometry, FP32 quadrature nodes).
//
// Translation operators (Sec. 2.3, Eq. 11-14).  Expansions use the addition theorem
//   G(x,y) = i k sum_{n,m} h_n(k r_x) Y_nm(x^) j_n(k r_y) conj(Y_nm(y^)),  r_y < r_x,
// with orthonormal Y_nm = Q_n^|m|(cos t) e^{i m phi} (no Condon-Shortley phase in
// this library) and level scaling s = min(1, k a): jt_n = j_n / s^n,
// ht_n = h_n s^(n+1).  With the pre-scaled density sh_j = k w_j s_j / (4 pi):
//   multipole  M_nm = sum_j sh_j jt_n(k r_j) conj(Y_nm)  ->  phi(x) = (4 pi i / s) sum M_nm ht_n Y_nm
//   local      phi(x) = sum_nm L_nm jt_n(k r) Y_nm
// Every operator maps coefficients of one basis family to another; its entries
// are inner products with the orthonormal Y on a sphere of radius rho about the
// new centre, divided by jt_n(k rho).  They are evaluated here with a product
// rule (Gauss-Legendre in cos t, uniform in phi) as a batched complex GEMM.
//
// Self/near correction (Sec. 2.2, Listing 1): for target x_i and each triangle in
// its singular set, int_T G(x_i,y) L_a(y) dS_y by a Duffy-type collapse about the
// point of T nearest to x_i, with a sinh grading of the edge coordinate (and of
// the radius when x_i is off the triangle), minus the point-rule term (FP64) that
// the FMM already added.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <vector>

#include "hfmm_internal.cuh"

namespace hfmm {

static constexpr double kPi = 3.14159265358979323846;

// ============================================================== host special functions
void host_jn_scaled(int nmax, double z, double s, double* out) {
    if (z == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
        return;
    }
    if (z < 2.0) {
        double lead = 1.0;  // (z/s)^n / (2n+1)!!
        for (int n = 0; n <= nmax; ++n) {
            if (n) lead *= (z / s) / (2 * n + 1);
            double term = 1.0, sum = 1.0;
            for (int q = 1; q < 60; ++q) {
                term *= -0.5 * z * z / (q * (2.0 * n + 2.0 * q + 1.0));
                sum += term;
                if (std::fabs(term) <= 1e-17 * std::fabs(sum)) break;
            }
            out[n] = lead * sum;
        }
        return;
    }
    // backward recurrence from well above max(nmax, z)
    int top = nmax + 32 + (int)z;
    double fn1 = 0.0, fn = 1e-200;
    for (int n = top; n > nmax; --n) {
        double f = (2.0 * n + 1.0) / z * fn - fn1;
        fn1 = fn;
        fn = f;
        if (std::fabs(fn) > 1e200) { fn *= 1e-200; fn1 *= 1e-200; }
    }
    // fn = f_nmax, fn1 = f_{nmax+1}
    out[nmax] = fn;
    double up = fn1;
    for (int n = nmax; n >= 1; --n) {
        double f = (2.0 * n + 1.0) / z * out[n] - up;
        up = out[n];
        out[n - 1] = f;
        if (std::fabs(f) > 1e200) {
            for (int m = n - 1; m <= nmax; ++m) out[m] *= 1e-200;
            up *= 1e-200;
        }
    }
    double j0 = std::sin(z) / z, j1 = std::sin(z) / (z * z) - std::cos(z) / z;
    double c = std::fabs(j0) > std::fabs(j1) ? j0 / out[0] : j1 / out[1];
    double sp = 1.0;
    for (int n = 0; n <= nmax; ++n) {
        out[n] *= c / sp;
        sp *= s;
    }
}

void host_hn_scaled(int nmax, double z, double s, double* re, double* im) {
    host_jn_scaled(nmax, z, s, re);
    double s2 = s;  // s^(2n+1)
    for (int n = 0; n <= nmax; ++n) {
        re[n] *= s2;
        s2 *= s * s;
    }
    double y0 = -std::cos(z) / z * s;
    double y1 = (-std::cos(z) / (z * z) - std::sin(z) / z) * s * s;
    im[0] = y0;
    if (nmax >= 1) im[1] = y1;
    for (int n = 2; n <= nmax; ++n) im[n] = (2.0 * n - 1.0) * (s / z) * im[n - 1] - s * s * im[n - 2];
}

// ============================================================== device special functions
__device__ static void d_jn_scaled(int nmax, double z, double s, double* out) {
    if (z == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
        return;
    }
    if (z < 2.0) {
        double lead = 1.0;
        for (int n = 0; n <= nmax; ++n) {
            if (n) lead *= (z / s) / (2 * n + 1);
            double term = 1.0, sum = 1.0;
            for (int q = 1; q < 60; ++q) {
                term *= -0.5 * z * z / (q * (2.0 * n + 2.0 * q + 1.0));
                sum += term;
                if (fabs(term) <= 1e-17 * fabs(sum)) break;
            }
            out[n] = lead * sum;
        }
        return;
    }
    int top = nmax + 32 + (int)z;
    double fn1 = 0.0, fn = 1e-200;
    for (int n = top; n > nmax; --n) {
        double f = (2.0 * n + 1.0) / z * fn - fn1;
        fn1 = fn;
        fn = f;
        if (fabs(fn) > 1e200) { fn *= 1e-200; fn1 *= 1e-200; }
    }
    out[nmax] = fn;
    double up = fn1;
    for (int n = nmax; n >= 1; --n) {
        double f = (2.0 * n + 1.0) / z * out[n] - up;
        up = out[n];
        out[n - 1] = f;
        if (fabs(f) > 1e200) {
            for (int m = n - 1; m <= nmax; ++m) out[m] *= 1e-200;
            up *= 1e-200;
        }
    }
    double j0 = sin(z) / z, j1 = sin(z) / (z * z) - cos(z) / z;
    double c = fabs(j0) > fabs(j1) ? j0 / out[0] : j1 / out[1];
    double sp = 1.0;
    for (int n = 0; n <= nmax; ++n) {
        out[n] *= c / sp;
        sp *= s;
    }
}

// radial part of the translated functions: type 0 jt_n, type 1 (4 pi i / s) ht_n
__device__ static void d_radial(int type, int nmax, double z, double s, double2* out) {
    double jr[HFMM_PMAX + 1];
    d_jn_scaled(nmax, z, s, jr);
    if (type == 0) {
        for (int n = 0; n <= nmax; ++n) out[n] = make_double2(jr[n], 0.0);
        return;
    }
    double s2 = s, ym2 = 0.0, ym1 = 0.0;
    double c = 4.0 * kPi / s;
    for (int n = 0; n <= nmax; ++n) {
        double y;
        if (n == 0) y = -cos(z) / z * s;
        else if (n == 1) y = (-cos(z) / (z * z) - sin(z) / z) * s * s;
        else y = (2.0 * n - 1.0) * (s / z) * ym1 - s * s * ym2;
        ym2 = ym1;
        ym1 = y;
        double hre = jr[n] * s2;
        s2 *= s * s;
        // (4 pi i / s) (hre + i y) = (4 pi / s) (-y + i hre)
        out[n] = make_double2(-c * y, c * hre);
    }
}

// ============================================================== projection kernels
// E[op][q][j] = f_j(rho s_q - d0[op]),  j = n*n+n+m
__global__ void k_proj_eval(int type, int pf, double sf, double k, double rho, int nth, int nph,
                            const double* __restrict__ ct_nodes, const double* __restrict__ d0, int nops,
                            double2* __restrict__ E) {
    int64_t Q = (int64_t)nth * nph;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Q * nops) return;
    int op = (int)(idx / Q);
    int64_t q = idx % Q;
    int it = (int)(q / nph), ip = (int)(q % nph);
    double ct = ct_nodes[it], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * kPi * ip / nph;
    double y0 = rho * st * cos(ph) - d0[3 * op], y1 = rho * st * sin(ph) - d0[3 * op + 1],
           y2 = rho * ct - d0[3 * op + 2];
    double r = sqrt(y0 * y0 + y1 * y1 + y2 * y2);
    double2 rad[HFMM_PMAX + 1];
    d_radial(type, pf, k * r, sf, rad);
    double cth = 1.0, sth = 0.0, ex = 1.0, ey = 0.0;
    if (r > 0.0) {
        cth = y2 / r;
        double rxy = sqrt(y0 * y0 + y1 * y1);
        sth = rxy / r;
        if (rxy > 0.0) { ex = y0 / rxy; ey = y1 / rxy; }
    }
    int Pf = (pf + 1) * (pf + 1);
    double2* row = E + ((int64_t)op * Q + q) * Pf;
    double qmm = 0.28209479177387814;  // 1/sqrt(4 pi)
    double emr = 1.0, emi = 0.0;       // e^{i m phi}
    for (int m = 0; m <= pf; ++m) {
        if (m > 0) {
            qmm *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * sth;
            double t = emr * ex - emi * ey;
            emi = emr * ey + emi * ex;
            emr = t;
        }
        double qa = qmm, qb = 0.0;
        for (int n = m; n <= pf; ++n) {
            double qn;
            if (n == m) qn = qmm;
            else if (n == m + 1) qn = sqrt(2.0 * m + 3.0) * cth * qmm;
            else {
                double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
                double b = sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
                qn = a * (cth * qa - b * qb);
            }
            if (n > m) { qb = qa; qa = qn; }
            double2 R = rad[n];
            // R * qn * e^{+i m phi}
            double yr = qn * emr, yi = qn * emi;
            row[n * n + n + m] = make_double2(R.x * yr - R.y * yi, R.x * yi + R.y * yr);
            if (m > 0) row[n * n + n - m] = make_double2(R.x * yr + R.y * yi, -R.x * yi + R.y * yr);
        }
    }
}

// Bw[i][q] = w_q conj(Y_i(s_q)) / jt_{n_i}(k rho)
__global__ void k_proj_basis(int pb, int nth, int nph, const double* __restrict__ ct_nodes,
                             const double* __restrict__ ct_w, const double* __restrict__ inv_j,
                             double2* __restrict__ Bw) {
    int64_t Q = (int64_t)nth * nph;
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    int it = (int)(q / nph), ip = (int)(q % nph);
    double ct = ct_nodes[it], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * kPi * ip / nph;
    double wq = ct_w[it] * 2.0 * kPi / nph;
    double ex = cos(ph), ey = sin(ph);
    double qmm = 0.28209479177387814;
    double emr = 1.0, emi = 0.0;
    for (int m = 0; m <= pb; ++m) {
        if (m > 0) {
            qmm *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
            double t = emr * ex - emi * ey;
            emi = emr * ey + emi * ex;
            emr = t;
        }
        double qa = qmm, qb = 0.0;
        for (int n = m; n <= pb; ++n) {
            double qn;
            if (n == m) qn = qmm;
            else if (n == m + 1) qn = sqrt(2.0 * m + 3.0) * ct * qmm;
            else {
                double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
                double b = sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
                qn = a * (ct * qa - b * qb);
            }
            if (n > m) { qb = qa; qa = qn; }
            double c = wq * qn * inv_j[n];
            // conj(Y_{n,m}) = qn e^{-i m phi};  conj(Y_{n,-m}) = qn e^{+i m phi}
            Bw[(int64_t)(n * n + n + m) * Q + q] = make_double2(c * emr, -c * emi);
            if (m > 0) Bw[(int64_t)(n * n + n - m) * Q + q] = make_double2(c * emr, c * emi);
        }
    }
}

// T[op][i][j] = sum_q Bw[i][q] E[op][q][j]; out row-major [Pb][Pf], out2 = T^H [Pf][Pb]
__global__ void k_proj_gemm(int Pb, int Pf, int64_t Q, const double2* __restrict__ Bw,
                            const double2* __restrict__ E, float2* __restrict__ out,
                            float2* __restrict__ out2) {
    __shared__ double2 sa[16][17];
    __shared__ double2 sb[16][17];
    int op = blockIdx.z;
    int i = blockIdx.y * 16 + threadIdx.y;
    int j = blockIdx.x * 16 + threadIdx.x;
    const double2* Eo = E + (int64_t)op * Q * Pf;
    double re = 0.0, im = 0.0;
    for (int64_t q0 = 0; q0 < Q; q0 += 16) {
        int ai = blockIdx.y * 16 + threadIdx.y;
        int64_t aq = q0 + threadIdx.x;
        sa[threadIdx.y][threadIdx.x] = (ai < Pb && aq < Q) ? Bw[(int64_t)ai * Q + aq] : make_double2(0, 0);
        int64_t bq = q0 + threadIdx.y;
        int bj = blockIdx.x * 16 + threadIdx.x;
        sb[threadIdx.y][threadIdx.x] = (bj < Pf && bq < Q) ? Eo[bq * Pf + bj] : make_double2(0, 0);
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            double2 a = sa[threadIdx.y][t], b = sb[t][threadIdx.x];
            re += a.x * b.x - a.y * b.y;
            im += a.x * b.y + a.y * b.x;
        }
        __syncthreads();
    }
    if (i < Pb && j < Pf) {
        out[(int64_t)op * Pb * Pf + (int64_t)i * Pf + j] = make_float2((float)re, (float)im);
        if (out2) out2[(int64_t)op * Pb * Pf + (int64_t)j * Pb + i] = make_float2((float)re, (float)-im);
    }
}

// The same product in double-float arithmetic on the FP32 pipes (GB300's FP64 rate is a
// small fraction of its FP32 rate): each FP64 input is split into an FP32 pair hi + lo, every
// real multiply-add is an error-free product (hi * hi and its FMA residual, plus the two
// cross terms) added with Knuth's two-sum, so the accumulators keep about 48 significant
// bits; the result is rounded to FP32 like the FP64 kernel's.  Inputs or products beyond FP32's
// range give a non-finite value; the caller then repeats the batch with the FP64 kernel.
__device__ __forceinline__ void df_mad(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(sh, p);
    const float bb = __fsub_rn(t, sh);
    float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    err = __fadd_rn(err, __fadd_rn(sl, e));
    sh = __fadd_rn(t, err);
    sl = __fsub_rn(err, __fsub_rn(sh, t));
}

__device__ __forceinline__ float4 df_split2(double2 v) {  // (re_hi, re_lo, im_hi, im_lo)
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

__global__ void k_proj_gemm_df(int Pb, int Pf, int64_t Q, const double2* __restrict__ Bw,
                               const double2* __restrict__ E, float2* __restrict__ out,
                               float2* __restrict__ out2) {
    __shared__ float4 sa[16][17];
    __shared__ float4 sb[16][17];
    const int op = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y;
    const int j = blockIdx.x * 16 + threadIdx.x;
    const double2* Eo = E + (int64_t)op * Q * Pf;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int64_t q0 = 0; q0 < Q; q0 += 16) {
        const int ai = blockIdx.y * 16 + threadIdx.y;
        const int64_t aq = q0 + threadIdx.x;
        sa[threadIdx.y][threadIdx.x] = df_split2((ai < Pb && aq < Q) ? Bw[(int64_t)ai * Q + aq] : make_double2(0, 0));
        const int64_t bq = q0 + threadIdx.y;
        const int bj = blockIdx.x * 16 + threadIdx.x;
        sb[threadIdx.y][threadIdx.x] = df_split2((bj < Pf && bq < Q) ? Eo[bq * Pf + bj] : make_double2(0, 0));
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
            const float4 a = sa[threadIdx.y][t], b = sb[t][threadIdx.x];
            df_mad(rh, rl, a.x, a.y, b.x, b.y);     // + Re a Re b
            df_mad(rh, rl, -a.z, -a.w, b.z, b.w);   // - Im a Im b
            df_mad(ih, il, a.x, a.y, b.z, b.w);     // + Re a Im b
            df_mad(ih, il, a.z, a.w, b.x, b.y);     // + Im a Re b
        }
        __syncthreads();
    }
    if (i < Pb && j < Pf) {
        const float re = __fadd_rn(rh, rl), im = __fadd_rn(ih, il);
        out[(int64_t)op * Pb * Pf + (int64_t)i * Pf + j] = make_float2(re, im);
        if (out2) out2[(int64_t)op * Pb * Pf + (int64_t)j * Pb + i] = make_float2(re, -im);
    }
}

// *bad = 1 if any of the n entries is not finite (grid-stride)
__global__ void k_any_nonfinite(const float2* __restrict__ a, int64_t n, int* __restrict__ bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[e].x) || !isfinite(a[e].y)) *bad = 1;
}

static void gauss_legendre_host(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void build_projection_ops(const ProjectionJob& job, double k, cudaStream_t st) {
    int Pf = (job.pf + 1) * (job.pf + 1), Pb = (job.pb + 1) * (job.pb + 1);
    int64_t Q = (int64_t)job.nth * job.nph;
    std::vector<double> gx, gw;
    gauss_legendre_host(job.nth, gx, gw);
    std::vector<double> jb(job.pb + 1), inv(job.pb + 1);
    host_jn_scaled(job.pb, k * job.rho, job.sb, jb.data());
    for (int n = 0; n <= job.pb; ++n) inv[n] = 1.0 / jb[n];
    DBuf<double> d_gx, d_gw, d_inv, d_d0;
    d_gx.upload(gx, nullptr, st);
    d_gw.upload(gw, nullptr, st);
    d_inv.upload(inv, nullptr, st);
    std::vector<double> d0(job.d0, job.d0 + 3 * (size_t)job.nops);
    d_d0.upload(d0, nullptr, st);
    DBuf<double2> Bw;
    Bw.alloc((size_t)Pb * Q, nullptr);
    k_proj_basis<<<(unsigned)((Q + 127) / 128), 128, 0, st>>>(job.pb, job.nth, job.nph, d_gx.p, d_gw.p,
                                                               d_inv.p, Bw.p);
    HFMM_CUDA(cudaGetLastError());
    // batch operators so the evaluated functions stay under ~512 MB
    int64_t per_op = Q * Pf * (int64_t)sizeof(double2);
    int batch = (int)std::max<int64_t>(1, std::min<int64_t>(job.nops, (512ll << 20) / per_op));
    DBuf<double2> E;
    E.alloc((size_t)batch * Q * Pf, nullptr);
    DBuf<int> bad;
    bad.alloc(1, nullptr);
    // HFMM_PROJECTION_FP64=1 forces the FP64 kernel (the reference the double-float one is tested against)
    const char* env = std::getenv("HFMM_PROJECTION_FP64");
    const bool fp64_only = env && env[0] == '1';
    for (int o0 = 0; o0 < job.nops; o0 += batch) {
        int nb = std::min(batch, job.nops - o0);
        int64_t nthreads = Q * nb;
        k_proj_eval<<<(unsigned)((nthreads + 127) / 128), 128, 0, st>>>(
            job.type, job.pf, job.sf, k, job.rho, job.nth, job.nph, d_gx.p, d_d0.p + 3 * o0, nb, E.p);
        HFMM_CUDA(cudaGetLastError());
        dim3 grid((Pf + 15) / 16, (Pb + 15) / 16, nb);
        float2* o = job.out + (int64_t)o0 * Pb * Pf;
        float2* o2 = job.out2 ? job.out2 + (int64_t)o0 * Pb * Pf : nullptr;
        bool redo = fp64_only;
        if (!fp64_only) {
            k_proj_gemm_df<<<grid, dim3(16, 16), 0, st>>>(Pb, Pf, Q, Bw.p, E.p, o, o2);
            HFMM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            const int64_t n = (int64_t)nb * Pb * Pf;
            k_any_nonfinite<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(o, n, bad.p);
            HFMM_CUDA(cudaGetLastError());
            int h_bad = 0;
            HFMM_CUDA(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            HFMM_CUDA(cudaStreamSynchronize(st));
            redo = h_bad != 0;
        }
        if (redo) k_proj_gemm<<<grid, dim3(16, 16), 0, st>>>(Pb, Pf, Q, Bw.p, E.p, o, o2);
        HFMM_CUDA(cudaGetLastError());
    }
    HFMM_CUDA(cudaStreamSynchronize(st));  // scratch buffers are freed on return
}

// ============================================================== M2L operators by reflection
// Reflecting the whole configuration in a coordinate plane maps the basis functions
// b_{n,m} = (radial) Q_n^|m|(cos t) e^{i m phi} onto signed basis functions of the same
// degree: x -> -x gives (-1)^m b_{n,-m}, y -> -y gives b_{n,-m}, z -> -z gives
// (-1)^{n+m} b_{n,m}. Both expansion kinds transform alike, so for a composition R of such
// flips  T(R d)[c][c'] = s(c) s(c') T(d)[mu(c)][mu(c')],  with s the product of the signs
// and mu(m) = -m when exactly one of the x, y flips is present. Only the offsets with
// non-negative components are projected; the others follow exactly.
__global__ void k_expand_reflections(const float2* __restrict__ canon, int P, int nops, const int4* __restrict__ map,
                                     float2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int op = blockIdx.y;
    if (e >= (int64_t)P * P || op >= nops) return;
    const int4 mp = map[op];  // (canonical operator, flip x, flip y, flip z)
    const int c = (int)(e / P), cp = (int)(e % P);
    auto xf = [&](int q, int& mu, int& sgn) {
        int n = (int)sqrtf((float)q);
        while (n * n > q) --n;
        while ((n + 1) * (n + 1) <= q) ++n;
        const int m = q - n * n - n;
        sgn = 1;
        if (mp.y && (m & 1)) sgn = -sgn;
        if (mp.w && ((n + m) & 1)) sgn = -sgn;
        const int m2 = (mp.y != mp.z) ? -m : m;
        mu = n * n + n + m2;
    };
    int mu, s1, mu2, s2;
    xf(c, mu, s1);
    xf(cp, mu2, s2);
    const float2 v = canon[(int64_t)mp.x * P * P + (int64_t)mu * P + mu2];
    const float sg = (float)(s1 * s2);
    out[(int64_t)op * P * P + e] = make_float2(sg * v.x, sg * v.y);
}

void expand_m2l_reflections(const float2* canon, int P, int nops, const int4* map, float2* out, cudaStream_t st) {
    const int64_t n = (int64_t)P * P;
    k_expand_reflections<<<dim3((unsigned)((n + 255) / 256), (unsigned)nops), 256, 0, st>>>(canon, P, nops, map, out);
    HFMM_CUDA(cudaGetLastError());
}

// ============================================================== self / near correction
struct d3 {
    double x, y, z;
};
__device__ __forceinline__ d3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double nrm(d3 a) { return sqrt(dot(a, a)); }

// closest point of triangle (a,b,c) to p, all in one plane
__device__ static d3 closest_on_triangle(d3 p, d3 a, d3 b, d3 c) {
    d3 ab = b - a, ac = c - a, ap = p - a;
    double d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0 && d2 <= 0) return a;
    d3 bp = p - b;
    double d3_ = dot(ab, bp), d4 = dot(ac, bp);
    if (d3_ >= 0 && d4 <= d3_) return b;
    double vc = d1 * d4 - d3_ * d2;
    if (vc <= 0 && d1 >= 0 && d3_ <= 0) return a + (d1 / (d1 - d3_)) * ab;
    d3 cp = p - c;
    double d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0 && d5 <= d6) return c;
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0 && d2 >= 0 && d6 <= 0) return a + (d2 / (d2 - d6)) * ac;
    double va = d3_ * d6 - d5 * d4;
    if (va <= 0 && (d4 - d3_) >= 0 && (d5 - d6) >= 0) return b + ((d4 - d3_) / ((d4 - d3_) + (d5 - d6))) * (c - b);
    double den = 1.0 / (va + vb + vc);
    return a + (vb * den) * ab + (vc * den) * ac;
}

template <typename T>
struct v3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ v3<T> cv(d3 a) {
    return {(T)a.x, (T)a.y, (T)a.z};
}
__device__ __forceinline__ void sc(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sc(double a, double* s, double* c) { sincos(a, s, c); }

// out[a] = int_T G(x,y) (2 lambda_a(y) - 1/3) dS_y
//
// The geometry of each sub-triangle (nearest point, edge frame, the limits of the
// sinh-graded edge coordinate) is taken in FP64; the 3 nq^2 quadrature nodes run in T in
// coordinates relative to x (lengths of the order of the mesh size, so the node positions
// keep T's relative precision), each row of nq nodes summed in T and the rows in FP64.  With
// T = float every node term is positive apart from the phase, so the integrals carry about
// 1e-6 relative error against 1e-7 for FP32 storage; T = double (the accurate operator)
// leaves the rule's own error.
template <typename T>
__device__ static void tri_integrals(d3 x, d3 v0, d3 v1, d3 v2, double k, bool self, int nq,
                                     const T* gx, const T* gw, double2 out[3]) {
    d3 nn = cross(v1 - v0, v2 - v0);
    double twoA = nrm(nn);
    d3 nh = (1.0 / twoA) * nn;
    d3 g[3] = {(1.0 / twoA) * cross(nh, v2 - v1), (1.0 / twoA) * cross(nh, v0 - v2),
               (1.0 / twoA) * cross(nh, v1 - v0)};
    double w = dot(x - v0, nh);
    d3 xp = x - w * nh;
    d3 pc = self ? xp : closest_on_triangle(xp, v0, v1, v2);
    double delta = self ? 0.0 : nrm(x - pc);
    d3 vv[3] = {v0, v1, v2};
    double acc_r[3] = {0, 0, 0}, acc_i[3] = {0, 0, 0};
    // node-loop constants: positions relative to x, barycentric gradients
    const v3<T> pcx = cv<T>(pc - x), pcv = cv<T>(pc - v0);
    const v3<T> gf[3] = {cv<T>(g[0]), cv<T>(g[1]), cv<T>(g[2])};
    const T kf = (T)k, deltaf = (T)delta;
    const T inv4pi = (T)(1.0 / (4.0 * kPi));
    for (int e = 0; e < 3; ++e) {
        d3 a = vv[e], b = vv[(e + 1) % 3];
        d3 ed = b - a;
        double len = nrm(ed);
        d3 lh = (1.0 / len) * ed;
        d3 am = a - pc;
        double lm = dot(am, lh), lp = dot(b - pc, lh);
        d3 perp = am - lm * lh;  // from pc to the foot on the edge line
        double de = nrm(perp);
        if (de <= 1e-12 * len) continue;  // pc on this edge: empty sub-triangle
        double s0 = asinh(lm / de), s1 = asinh(lp / de);
        const T s0f = (T)s0, dsf = (T)(s1 - s0), def = (T)de;
        const v3<T> pf = cv<T>(perp), lf = cv<T>(lh);
        for (int iq = 0; iq < nq; ++iq) {
            const T s = s0f + dsf * gx[iq];
            const T ws = dsf * gw[iq];
            const T l = def * sinh(s);
            const v3<T> E = {pf.x + l * lf.x, pf.y + l * lf.y, pf.z + l * lf.z};
            const T En = sqrt(E.x * E.x + E.y * E.y + E.z * E.z);  // = de cosh(s) = dl/ds
            const T tmax_tau = delta > 0.0 ? asinh(En / deltaf) : (T)1;
            const T rowc = def * En * ws;
            T rr[3] = {0, 0, 0}, ri[3] = {0, 0, 0};
            for (int jq = 0; jq < nq; ++jq) {
                T t, wt;
                if (delta > 0.0) {
                    const T tau = tmax_tau * gx[jq];
                    const T q = deltaf / En;
                    t = q * sinh(tau);
                    wt = tmax_tau * gw[jq] * q * cosh(tau);
                } else {
                    t = gx[jq];
                    wt = gw[jq];
                }
                // y - x and y - v0 for y = pc + t E
                const v3<T> yx = {pcx.x + t * E.x, pcx.y + t * E.y, pcx.z + t * E.z};
                const v3<T> yv = {pcv.x + t * E.x, pcv.y + t * E.y, pcv.z + t * E.z};
                const T R = sqrt(yx.x * yx.x + yx.y * yx.y + yx.z * yx.z);
                // dS = t * de * dl * dt = t * de * En * ds * dt
                T sn, cs;
                sc(kf * R, &sn, &cs);
                const T f = t * rowc * wt * inv4pi / R;
                const T lam[3] = {(T)1 + gf[0].x * yv.x + gf[0].y * yv.y + gf[0].z * yv.z,
                                  gf[1].x * yv.x + gf[1].y * yv.y + gf[1].z * yv.z,
                                  gf[2].x * yv.x + gf[2].y * yv.y + gf[2].z * yv.z};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const T L = (T)2 * lam[q] - (T)1 / (T)3;
                    rr[q] += f * cs * L;
                    ri[q] += f * sn * L;
                }
            }
            for (int q = 0; q < 3; ++q) {
                acc_r[q] += (double)rr[q];
                acc_i[q] += (double)ri[q];
            }
        }
    }
    for (int q = 0; q < 3; ++q) out[q] = make_double2(acc_r[q], acc_i[q]);
}

__device__ static int64_t find_key(const uint64_t* keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        uint64_t v = keys[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}
__device__ __forceinline__ uint64_t dmorton(int64_t x, int64_t y, int64_t z) {
    return (spread3((uint64_t)x) << 2) | (spread3((uint64_t)y) << 1) | spread3((uint64_t)z);
}

// near/self triangle set of sorted point i (sorted ascending, own triangle included)
__device__ static int near_set(const CorrInputs& in, int64_t i, int32_t* list, int* overflow) {
    int cnt = 0;
    list[cnt++] = in.tri_s[i];
    int4 c = in.pt_ijk[i];
    int sh = in.L - in.search_level;
    int64_t cx = c.x >> sh, cy = c.y >> sh, cz = c.z >> sh;
    int64_t nl = (int64_t)1 << in.search_level;
    double xi = in.x64s[3 * i], yi = in.x64s[3 * i + 1], zi = in.x64s[3 * i + 2];
    double r2 = in.r_near * in.r_near;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t bx = cx + dx, by = cy + dy, bz = cz + dz;
                if (bx < 0 || by < 0 || bz < 0 || bx >= nl || by >= nl || bz >= nl) continue;
                int64_t b = find_key(in.skey, in.nsbox, dmorton(bx, by, bz));
                if (b < 0) continue;
                for (int32_t j = in.sstart[b]; j < in.sstart[b + 1]; ++j) {
                    double ex = xi - in.x64s[3 * j], ey = yi - in.x64s[3 * j + 1], ez = zi - in.x64s[3 * j + 2];
                    if (ex * ex + ey * ey + ez * ez > r2) continue;
                    int32_t t = in.tri_s[j];
                    bool seen = false;
                    for (int q = 0; q < cnt; ++q) seen |= (list[q] == t);
                    if (seen) continue;
                    if (cnt < HFMM_NEAR_CAP) list[cnt++] = t;
                    else *overflow = 1;
                }
            }
    // insertion sort for a deterministic column order
    for (int a = 1; a < cnt; ++a) {
        int32_t v = list[a];
        int b = a - 1;
        while (b >= 0 && list[b] > v) { list[b + 1] = list[b]; --b; }
        list[b + 1] = v;
    }
    return cnt;
}

__global__ void k_corr_count(CorrInputs in, int64_t* __restrict__ rowptr, int* __restrict__ overflow) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in.N) return;
    int32_t list[HFMM_NEAR_CAP];
    int c = near_set(in, i, list, overflow);
    rowptr[i + 1] = 3 * (int64_t)c;
}

__global__ void k_corr_fill(CorrInputs in, const double* __restrict__ gx, const double* __restrict__ gw,
                            const int64_t* __restrict__ rowptr, int32_t* __restrict__ col,
                            float2* __restrict__ val, double2* __restrict__ val64, int* __restrict__ overflow) {
    __shared__ double sgx[64], sgw[64];  // the rule on [0, 1] (quad_order <= 64)
    __shared__ float sgxf[64], sgwf[64];
    for (int q = threadIdx.x; q < in.quad_order; q += blockDim.x) {
        sgx[q] = gx[q];
        sgw[q] = gw[q];
        sgxf[q] = (float)gx[q];
        sgwf[q] = (float)gw[q];
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in.N) return;
    int32_t list[HFMM_NEAR_CAP];
    int c = near_set(in, i, list, overflow);
    d3 x = mk(in.x64s[3 * i], in.x64s[3 * i + 1], in.x64s[3 * i + 2]);
    int64_t o = rowptr[i];
    int32_t own = in.tri_s[i];
    for (int q = 0; q < c; ++q) {
        int32_t n = list[q];
        d3 v[3];
        for (int a = 0; a < 3; ++a) {
            int32_t vi = in.F[3 * (int64_t)n + a];
            v[a] = mk(in.V[3 * (int64_t)vi], in.V[3 * (int64_t)vi + 1], in.V[3 * (int64_t)vi + 2]);
        }
        double2 I3[3];
        if (val64)  // the accurate operator: FP64 nodes
            tri_integrals<double>(x, v[0], v[1], v[2], in.k, n == own, in.quad_order, sgx, sgw, I3);
        else
            tri_integrals<float>(x, v[0], v[1], v[2], in.k, n == own, in.quad_order, sgxf, sgwf, I3);
        for (int a = 0; a < 3; ++a) {
            int32_t js = in.iperm[3 * (int64_t)n + a];
            double re = I3[a].x, im = I3[a].y;
            double wj = in.w64s[js];
            if (js != i) {
                // remove the point-rule term w_j G(x_i, x_j) that the FMM adds
                double ex = x.x - in.x64s[3 * js], ey = x.y - in.x64s[3 * js + 1], ez = x.z - in.x64s[3 * js + 2];
                double R = sqrt(ex * ex + ey * ey + ez * ez);
                double sn, cs;
                sincos(in.k * R, &sn, &cs);
                re -= wj * cs / (4.0 * kPi * R);
                im -= wj * sn / (4.0 * kPi * R);
            }
            // stored against the pre-scaled density k w_j s_j / (4 pi)
            double sc = 4.0 * kPi / (in.k * wj);
            col[o + a] = js;
            val[o + a] = make_float2((float)(re * sc), (float)(im * sc));
            if (val64) val64[o + a] = make_double2(re * sc, im * sc);
        }
        o += 3;
    }
}

int64_t build_correction(hfmm_plan* P, const CorrInputs& in, cudaStream_t st) {
    DBuf<int> ovf;
    ovf.alloc(1, nullptr);
    HFMM_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), st));
    P->corr_ptr.alloc(in.N + 1, &P->dev_bytes);
    HFMM_CUDA(cudaMemsetAsync(P->corr_ptr.p, 0, sizeof(int64_t), st));
    unsigned nb = (unsigned)((in.N + 127) / 128);
    k_corr_count<<<nb, 128, 0, st>>>(in, P->corr_ptr.p, ovf.p);
    HFMM_CUDA(cudaGetLastError());
    std::vector<int64_t> rp(in.N + 1);
    HFMM_CUDA(cudaMemcpyAsync(rp.data(), P->corr_ptr.p, sizeof(int64_t) * (in.N + 1), cudaMemcpyDeviceToHost, st));
    int h_ovf = 0;
    HFMM_CUDA(cudaMemcpyAsync(&h_ovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    if (h_ovf) throw HfmmError{HFMM_E_OVERFLOW, "near set larger than HFMM_NEAR_CAP triangles: lower near_factor"};
    rp[0] = 0;
    for (int64_t i = 0; i < in.N; ++i) rp[i + 1] += rp[i];
    int64_t nnz = rp[in.N];
    if (P->cfg.mem_budget_bytes > 0 &&
        (double)P->dev_bytes + (double)nnz * 12.0 > P->cfg.mem_budget_bytes)
        throw HfmmError{HFMM_E_NOMEM, "plan exceeds the configured device memory budget"};
    P->corr_ptr.upload(rp, nullptr, st);
    P->corr_col.alloc(nnz, &P->dev_bytes);
    P->corr_val.alloc(nnz, &P->dev_bytes);
    std::vector<double> gx, gw;
    gauss_legendre_host(in.quad_order, gx, gw);
    for (int q = 0; q < in.quad_order; ++q) {  // map to [0, 1]
        gx[q] = 0.5 * (gx[q] + 1.0);
        gw[q] *= 0.5;
    }
    DBuf<double> d_gx, d_gw;
    d_gx.upload(gx, nullptr, st);
    d_gw.upload(gw, nullptr, st);
    if (P->cfg.precision == 1) P->corr_val64.alloc(nnz, &P->dev_bytes);
    k_corr_fill<<<nb, 128, 0, st>>>(in, d_gx.p, d_gw.p, P->corr_ptr.p, P->corr_col.p, P->corr_val.p,
                                     P->cfg.precision == 1 ? P->corr_val64.p : nullptr, ovf.p);
    HFMM_CUDA(cudaGetLastError());
    HFMM_CUDA(cudaStreamSynchronize(st));
    return nnz;
}

}  // namespace hfmm
