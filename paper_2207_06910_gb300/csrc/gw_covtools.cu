// gw_covtools.cu -- per-event covariance tools on the Fisher matrices:
// eigensystem (CheckFisher, Sec. 4.1), covariance with the inversion options
// of CovMatr (Sec. 4.1) after fixParams / addPrior (Sec. 4.2), the sub-matrix
// of kept parameters (fixing on Gamma, marginalising on C) and the sky-
// localisation area Delta Omega_X% (Sec. 4.1).
//
// One thread per event; every matrix of a thread (at most 11 x 11 FP64) lives
// in its local memory.  These are small dense tools applied after the Fisher
// pass, FP64 throughout (the matrices reach condition numbers of 1e14).
#include <cmath>

#include "gw_kernels.cuh"

namespace gw {

namespace {

constexpr int CP = 11;   // largest parameter count

// packed upper-triangle index of (i, j), i <= j, row-major over P parameters
__device__ __forceinline__ int pk(int i, int j, int P)
{
    if (i > j) {
        const int t = i;
        i = j;
        j = t;
    }
    return i * P - i * (i - 1) / 2 + (j - i);
}

// cyclic Jacobi on a symmetric P x P matrix: A = V diag(w) V^T (A destroyed),
// V[i * P + k] = component i of eigenvector k; eigenpairs sorted by increasing
// w and each eigenvector's largest-magnitude component made positive
__device__ void jacobi_eigv(int P, double *A, double *w, double *V)
{
    for (int i = 0; i < P * P; i++) V[i] = 0.0;
    for (int i = 0; i < P; i++) V[i * P + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) {
                const double x = A[i * P + j] * A[i * P + j];
                tot += x;
                if (i != j) off += x;
            }
        if (!(off > 1e-34 * tot)) break;
        for (int p = 0; p < P; p++)
            for (int q = p + 1; q < P; q++) {
                const double apq = A[p * P + q];
                if (apq == 0.0) continue;
                const double tau = (A[q * P + q] - A[p * P + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < P; k++) {
                    const double akp = A[k * P + p], akq = A[k * P + q];
                    A[k * P + p] = c * akp - sn * akq;
                    A[k * P + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < P; k++) {
                    const double apk = A[p * P + k], aqk = A[q * P + k];
                    A[p * P + k] = c * apk - sn * aqk;
                    A[q * P + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < P; k++) {
                    const double vkp = V[k * P + p], vkq = V[k * P + q];
                    V[k * P + p] = c * vkp - sn * vkq;
                    V[k * P + q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < P; i++) w[i] = A[i * P + i];
    for (int a = 0; a < P; a++) {
        int m = a;
        for (int b = a + 1; b < P; b++)
            if (w[b] < w[m]) m = b;
        if (m != a) {
            double t = w[a];
            w[a] = w[m];
            w[m] = t;
            for (int i = 0; i < P; i++) {
                t = V[i * P + a];
                V[i * P + a] = V[i * P + m];
                V[i * P + m] = t;
            }
        }
    }
    for (int k = 0; k < P; k++) {
        int im = 0;
        for (int i = 1; i < P; i++)
            if (fabs(V[i * P + k]) > fabs(V[im * P + k])) im = i;
        if (V[im * P + k] < 0.0)
            for (int i = 0; i < P; i++) V[i * P + k] = -V[i * P + k];
    }
}

__global__ void k_fisher_eig(int64_t n, int P, int normalize, const double *F, double *w_out,
                             double *v_out)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double A[CP * CP], V[CP * CP], w[CP], d[CP];
    bool norm = normalize != 0;
    for (int i = 0; i < P; i++)
        if (!(F[(int64_t)pk(i, i, P) * n + e] > 0.0)) norm = false;
    for (int i = 0; i < P; i++) d[i] = norm ? sqrt(F[(int64_t)pk(i, i, P) * n + e]) : 1.0;
    for (int i = 0; i < P; i++)
        for (int j = 0; j < P; j++) A[i * P + j] = F[(int64_t)pk(i, j, P) * n + e] / (d[i] * d[j]);
    jacobi_eigv(P, A, w, V);
    if (w_out)
        for (int i = 0; i < P; i++) w_out[(int64_t)i * n + e] = w[i];
    if (v_out)
        for (int i = 0; i < P * P; i++) v_out[(int64_t)i * n + e] = V[i];
}

__global__ void k_covariance(CovArgs a, const double *F, double *cov, double *cond,
                             double *eps_out, int32_t *status)
{
    const int64_t n = a.n;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int P = a.P, K = a.Pk;
    double G[CP * CP], A[CP * CP], V[CP * CP], C[CP * CP], w[CP], d[CP];
    int st = 0;
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) {
            double g = F[(int64_t)pk(a.idx[i], a.idx[j], P) * n + e];
            if (i == j) g += a.prior[a.idx[i]];
            G[i * K + j] = g;
            if (!isfinite(g)) st |= 4;
        }
    const int npk = K * (K + 1) / 2;
    auto fail = [&](int bits, double kappa) {
        for (int q = 0; q < npk; q++) cov[(int64_t)q * n + e] = NAN;
        if (cond) cond[e] = kappa;
        if (eps_out) eps_out[e] = NAN;
        if (status) status[e] = bits;
    };
    if (st) {
        fail(st, NAN);
        return;
    }
    // normalisation by sqrt(diag) unless a diagonal element is not positive
    bool norm = true;
    for (int i = 0; i < K; i++)
        if (!(G[i * K + i] > 0.0)) norm = false;
    for (int i = 0; i < K; i++) d[i] = norm ? sqrt(G[i * K + i]) : 1.0;
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) A[i * K + j] = G[i * K + j] / (d[i] * d[j]);
    jacobi_eigv(K, A, w, V);
    double smax = 0.0, smin = INFINITY;
    for (int i = 0; i < K; i++) {
        smax = fmax(smax, fabs(w[i]));
        smin = fmin(smin, fabs(w[i]));
    }
    const double kappa = smin > 0.0 ? smax / smin : INFINITY;
    if (kappa > 1.0 / 2.220446049250313e-16) st |= 32;
    if (kappa > a.cond_max) {
        fail(st | 2, kappa);
        return;
    }
    bool use_svd = a.method >= 2 && a.method <= 4;
    if (a.method == 0 || a.method == 1) {
        // Cholesky of the normalised matrix in A (lower triangle), C = L^-T L^-1
        for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++) A[i * K + j] = G[i * K + j] / (d[i] * d[j]);
        bool pd = true;
        for (int j = 0; j < K && pd; j++) {
            double s = A[j * K + j];
            for (int k = 0; k < j; k++) s -= A[j * K + k] * A[j * K + k];
            if (!(s > 0.0)) {
                pd = false;
                break;
            }
            A[j * K + j] = sqrt(s);
            for (int i = j + 1; i < K; i++) {
                double t = A[i * K + j];
                for (int k = 0; k < j; k++) t -= A[i * K + k] * A[j * K + k];
                A[i * K + j] = t / A[j * K + j];
            }
        }
        if (!pd) {
            st |= 1;
            if (a.method == 0) {
                fail(st, kappa);
                return;
            }
            st |= 128;
            use_svd = true;
        } else {
            // L^-1 into the upper part of C (column c, rows i >= c), then C = L^-T L^-1
            double Li[CP * CP];
            for (int c = 0; c < K; c++)
                for (int i = c; i < K; i++) {
                    double t = (i == c) ? 1.0 : 0.0;
                    for (int k = c; k < i; k++) t -= A[i * K + k] * Li[k * K + c];
                    Li[i * K + c] = t / A[i * K + i];
                }
            for (int i = 0; i < K; i++)
                for (int j = i; j < K; j++) {
                    double t = 0.0;
                    for (int k = j; k < K; k++) t += Li[k * K + i] * Li[k * K + j];
                    C[i * K + j] = C[j * K + i] = t;
                }
        }
    }
    if (use_svd) {
        double iw[CP];
        const double floor_ = a.thresh * smax;
        for (int k = 0; k < K; k++) {
            const double s = fabs(w[k]);
            if (a.method == 3 && s < floor_) iw[k] = (w[k] < 0.0 ? -1.0 : 1.0) / floor_;
            else if (a.method == 4 && s < floor_) iw[k] = 0.0;
            else iw[k] = 1.0 / w[k];
        }
        for (int i = 0; i < K; i++)
            for (int j = i; j < K; j++) {
                double t = 0.0;
                for (int k = 0; k < K; k++) t += V[i * K + k] * iw[k] * V[j * K + k];
                C[i * K + j] = C[j * K + i] = t;
            }
    } else if (a.method == 5) {
        // LU with partial pivoting of the normalised matrix, columns of the inverse
        for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++) A[i * K + j] = G[i * K + j] / (d[i] * d[j]);
        int piv[CP];
        for (int i = 0; i < K; i++) piv[i] = i;
        bool sing = false;
        for (int k = 0; k < K && !sing; k++) {
            int m = k;
            for (int i = k + 1; i < K; i++)
                if (fabs(A[i * K + k]) > fabs(A[m * K + k])) m = i;
            if (A[m * K + k] == 0.0) {
                sing = true;
                break;
            }
            if (m != k) {
                for (int j = 0; j < K; j++) {
                    const double t = A[k * K + j];
                    A[k * K + j] = A[m * K + j];
                    A[m * K + j] = t;
                }
                const int t = piv[k];
                piv[k] = piv[m];
                piv[m] = t;
            }
            for (int i = k + 1; i < K; i++) {
                A[i * K + k] /= A[k * K + k];
                for (int j = k + 1; j < K; j++) A[i * K + j] -= A[i * K + k] * A[k * K + j];
            }
        }
        if (sing) {
            fail(st | 1, kappa);
            return;
        }
        for (int c = 0; c < K; c++) {
            double y[CP];
            for (int i = 0; i < K; i++) {
                double t = (piv[i] == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; k++) t -= A[i * K + k] * y[k];
                y[i] = t;
            }
            for (int i = K - 1; i >= 0; i--) {
                double t = y[i];
                for (int k = i + 1; k < K; k++) t -= A[i * K + k] * C[k * K + c];
                C[i * K + c] = t / A[i * K + i];
            }
        }
        // the LU inverse of a symmetric matrix is symmetric only to rounding:
        // inv_err is that of the full inverse, the packed output its upper
        // triangle
    }
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) C[i * K + j] /= d[i] * d[j];
    double eps = 0.0;
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) {
            double t = 0.0;
            for (int k = 0; k < K; k++) t = fma(G[i * K + k], C[k * K + j], t);
            eps = fmax(eps, fabs(t - (i == j ? 1.0 : 0.0)));
        }
    for (int i = 0; i < K; i++)
        for (int j = i; j < K; j++) cov[(int64_t)pk(i, j, K) * n + e] = C[i * K + j];
    if (cond) cond[e] = kappa;
    if (eps_out) eps_out[e] = eps;
    if (status) status[e] = st;
}

__global__ void k_submatrix(int64_t n, int P, int K, SubIdx s, const double *in, double *out)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    for (int i = 0; i < K; i++)
        for (int j = i; j < K; j++)
            out[(int64_t)pk(i, j, K) * n + e] = in[(int64_t)pk(s.idx[i], s.idx[j], P) * n + e];
}

__global__ void k_sky_area(int64_t n, int P, int it, int ip, const double *cov, const double *theta,
                           double lnq, double scale, double *area)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double ctt = cov[(int64_t)pk(it, it, P) * n + e];
    const double cpp = cov[(int64_t)pk(ip, ip, P) * n + e];
    const double ctp = cov[(int64_t)pk(it, ip, P) * n + e];
    const double det = fma(ctt, cpp, -ctp * ctp);
    area[e] = -2.0 * PI * fabs(sin(theta[e])) * sqrt(det) * lnq * scale;
}

// perturb_Fisher: Gamma'_ij = Gamma_ij (1 + eps r_ij) on the packed triangle
// (explicitly rounded operations: no contraction into an FMA)
__global__ void k_perturb(int64_t total, double eps, const double *F, const double *r, double *out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = __dmul_rn(F[q], __dadd_rn(1.0, __dmul_rn(eps, r[q])));
}

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_fisher_eig(int64_t n, int P, int normalize, const double *F, double *w,
                              double *V, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_fisher_eig<<<blocks_for(n, 128), 128, 0, s>>>(n, P, normalize, F, w, V);
    return cudaGetLastError();
}

cudaError_t launch_covariance(const CovArgs &a, const double *F, double *cov, double *cond,
                              double *eps, int32_t *status, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    k_covariance<<<blocks_for(a.n, 128), 128, 0, s>>>(a, F, cov, cond, eps, status);
    return cudaGetLastError();
}

cudaError_t launch_submatrix(int64_t n, int P, int K, const SubIdx &idx, const double *in,
                             double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_submatrix<<<blocks_for(n, 256), 256, 0, s>>>(n, P, K, idx, in, out);
    return cudaGetLastError();
}

cudaError_t launch_perturb(int64_t total, double eps, const double *F, const double *r,
                           double *out, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    int64_t nb = (total + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_perturb<<<(unsigned)nb, 256, 0, s>>>(total, eps, F, r, out);
    return cudaGetLastError();
}

cudaError_t launch_sky_area(int64_t n, int P, int it, int ip, const double *cov,
                            const double *theta, double perc, int units, double *area,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const double lnq = log1p(-perc / 100.0);
    const double scale = units == 1 ? (180.0 / PI) * (180.0 / PI) : 1.0;
    k_sky_area<<<blocks_for(n, 256), 256, 0, s>>>(n, P, it, ip, cov, theta, lnq, scale, area);
    return cudaGetLastError();
}

}  // namespace gw
