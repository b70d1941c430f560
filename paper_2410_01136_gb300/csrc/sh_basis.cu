// sh_basis.cu -- the low-order surrogate basis: real spherical harmonics at
// the HEALPix RING pixel centres, orthonormalised in their (l, m) order.
//
//   Y_l0 = Pbar_l0(z), Y_lm = sqrt(2) Pbar_lm(z) cos(m phi), Y_l,-m = sqrt(2)
//   Pbar_lm(z) sin(m phi) (m > 0), row l^2 + l + m, with Pbar_lm the
//   associated Legendre function normalised by sqrt((2l + 1)/(4 pi)
//   (l - m)!/(l + m)!) including the Condon-Shortley phase, from the standard
//   stable recurrences: Pbar_00 = 1/sqrt(4 pi), Pbar_mm = -sqrt((2m + 1)/(2m))
//   sin(theta) Pbar_m-1,m-1, Pbar_m+1,m = sqrt(2m + 3) z Pbar_mm, and
//   Pbar_lm = a_lm (z Pbar_l-1,m - b_lm Pbar_l-2,m) with
//   a_lm = sqrt((4 l^2 - 1)/(l^2 - m^2)), b_lm = sqrt(((l - 1)^2 - m^2)/(4 (l - 1)^2 - 1)).
// Sampled on the pixels the rows are nearly but not exactly orthogonal, so
// they are orthonormalised by CholeskyQR2 in FP64: E = L^-1 Y with
// Y Y^T = L L^T, twice.  Because L is lower triangular, E's first k rows span
// the first k harmonics for every k.  The dense linear algebra of this
// one-time set-up (Gram matrix, Cholesky factor, triangular solve) is cuBLAS
// and cuSOLVER.  The result is stored as BF16 hi + lo for the tensor-core
// projection.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include "march.cuh"

namespace synax {

__global__ void __launch_bounds__(128) k_sh_eval(double* __restrict__ Y, int nside, int npix, int n_basis, int lmax) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    Los<double> L;
    healpix_los<double>(nside, p, L);
    const double z = L.n[2];
    const double st = ::sqrt(fmax(0.0, (1.0 - z) * (1.0 + z)));
    const double phi = ::atan2(L.n[1], L.n[0]);
    double pmm = 0.28209479177387814;                  // 1 / sqrt(4 pi)
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) pmm *= -::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
        double sm = 0.0, cm = 1.0;
        if (m > 0) ::sincos(m * phi, &sm, &cm);
        const double rc = m > 0 ? 1.4142135623730951 * cm : 1.0, rs = 1.4142135623730951 * sm;
        double p2 = 0.0, p1 = pmm;                       // Pbar_{l-2,m}, Pbar_{l-1,m} as l advances
        for (int l = m; l <= lmax; ++l) {
            double pl;
            if (l == m) {
                pl = pmm;
            } else if (l == m + 1) {
                pl = ::sqrt(2.0 * m + 3.0) * z * pmm;
            } else {
                const double a = ::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                const double b = ::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                pl = a * (z * p1 - b * p2);
            }
            if (l > m) {
                p2 = p1;
                p1 = pl;
            }
            const int ip = l * l + l + m, in = l * l + l - m;
            if (ip < n_basis) Y[(long long)ip * npix + p] = pl * rc;
            if (m > 0 && in < n_basis) Y[(long long)in * npix + p] = pl * rs;
        }
    }
}

__global__ void k_to_bf16_hilo(const double* __restrict__ E, long long n, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = (float)E[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// Builds the orthonormal basis rows [n_basis][12 nside^2] as BF16 hi + lo, or
// copies them as FP64 to E_out when given (tests).  Synchronous.
int build_sh_basis(int nside, int n_basis, __nv_bfloat16* S_hi, __nv_bfloat16* S_lo, double* E_out) {
    const int npix = 12 * nside * nside;
    int lmax = 0;
    while ((lmax + 1) * (lmax + 1) < n_basis) ++lmax;
    double *Y = nullptr, *G = nullptr, *work = nullptr;
    int* info = nullptr;
    cublasHandle_t hb = nullptr;
    cusolverDnHandle_t hs = nullptr;
    int rc = SYNAX_OK;
    cudaError_t e = cudaMalloc(&Y, sizeof(double) * (size_t)n_basis * npix);
    if (e == cudaSuccess) e = cudaMalloc(&G, sizeof(double) * (size_t)n_basis * n_basis);
    if (e == cudaSuccess) e = cudaMalloc(&info, sizeof(int));
    if (e != cudaSuccess) rc = SYNAX_ENOMEM;
    if (rc == SYNAX_OK && (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS))
        rc = SYNAX_ECUDA;
    if (rc == SYNAX_OK) {
        k_sh_eval<<<(npix + 127) / 128, 128>>>(Y, nside, npix, n_basis, lmax);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = record_cuda_error((int)e);
    }
    int lwork = 0;
    if (rc == SYNAX_OK &&
        cusolverDnDpotrf_bufferSize(hs, CUBLAS_FILL_MODE_LOWER, n_basis, G, n_basis, &lwork) != CUSOLVER_STATUS_SUCCESS)
        rc = SYNAX_ECUDA;
    if (rc == SYNAX_OK && cudaMalloc(&work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)) != cudaSuccess)
        rc = SYNAX_ENOMEM;
    const double one = 1.0, zero = 0.0;
    // Y row-major [n_basis][npix] is A = Y^T column-major (npix x n_basis, lda npix)
    for (int pass = 0; pass < 2 && rc == SYNAX_OK; ++pass) {
        if (cublasDsyrk(hb, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, n_basis, npix, &one, Y, npix, &zero, G, n_basis) !=
                CUBLAS_STATUS_SUCCESS ||
            cusolverDnDpotrf(hs, CUBLAS_FILL_MODE_LOWER, n_basis, G, n_basis, work, lwork, info) !=
                CUSOLVER_STATUS_SUCCESS ||
            cublasDtrsm(hb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, npix, n_basis,
                        &one, G, n_basis, Y, npix) != CUBLAS_STATUS_SUCCESS) {
            rc = SYNAX_ECUDA;
            break;
        }
        int h_info = 0;
        e = cudaMemcpy(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = record_cuda_error((int)e);
        else if (h_info != 0) rc = SYNAX_EINVAL;          // not positive definite: n_basis beyond what the pixels resolve
    }
    if (rc == SYNAX_OK) {
        const long long n = (long long)n_basis * npix;
        if (S_hi && S_lo) k_to_bf16_hilo<<<1216, 256>>>(Y, n, S_hi, S_lo);
        e = cudaGetLastError();
        if (e == cudaSuccess && E_out) e = cudaMemcpy(E_out, Y, sizeof(double) * n, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = record_cuda_error((int)e);
    }
    if (hs) cusolverDnDestroy(hs);
    if (hb) cublasDestroy(hb);
    cudaFree(work);
    cudaFree(info);
    cudaFree(G);
    cudaFree(Y);
    return rc;
}

}  // namespace synax

extern "C" int synax_sh_basis(int nside, int n_basis, double* basis_dev) {
    if (nside < 1 || nside > 256 || (nside & (nside - 1)) || n_basis < 1 || n_basis > 12 * nside * nside ||
        !basis_dev)
        return SYNAX_EINVAL;
    return synax::build_sh_basis(nside, n_basis, nullptr, nullptr, basis_dev);
}
