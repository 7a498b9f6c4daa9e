// Complex score matrices (Section 4 of arXiv 2310.17556: complex SR, F = S^dagger S) solved
// natively on the two real planes of S = A + iB, stacked as Z = [A; B] (2n x m):
//
//   Gram      G = Z Z^T = [[A A^T, A B^T], [B A^T, B B^T]] gives W = S S^dagger + lambda I~ as
//             Re W = A A^T + B B^T + lambda I,  Im W = B A^T - A B^T = G21 - G21^T,
//             at 2 n^2 m real multiply-adds (the real 2n x 2m representation R(S) costs 4 n^2 m);
//   passes    S^dagger y and S u over Z with two real right-hand sides per complex one:
//               Re(S^dagger y) = Z^T [y_r; y_i],   Im(S^dagger y) = Z^T [y_i; -y_r],
//               S u = (A u_r - B u_i) + i (B u_r + A u_i) from the row sums Z [u_r, u_i],
//             so every pass reads each entry of A and B once (R(S) holds each twice);
//   n-space   the real 2n system R(W) [y_r; y_i] = [r_r; r_i], R(W) = [[Re W, -Im W], [Im W, Re W]]
//             (symmetric positive definite), factored and solved by the real kernels.
//
// The kernels here are the glue between those steps: the residual combine after a pass, the
// expansion of y into the pass's two columns per right-hand side, and the assembly of R(W).
// Layouts: a real n-space vector has rows 0..n-1 (real parts), n..2n-1 (imaginary parts), zero
// padding to n_pad; complex right-hand side q is pass column q (real part) and kc + q (imaginary).
#include "kernels.cuh"

namespace dfs {

namespace {

// r_real = R(S) u - lambda y from the pass partials P (parts x 2n x KQP, FP64, Z U per part):
//   r_r[i] = P[i][q] - P[n+i][kc+q] - lambda y_r[i],   r_i[i] = P[n+i][q] + P[i][kc+q] - lambda y_i[i]
// (without y: b = S v from the S v pass).  Parts are added in order (a fixed summation order).
// Writes R (FP64) and Zb (the solve type) with row stride KQN, zero in padding rows and columns.
// Also folds the pass's per-part stopping sums (U2part, parts x 2 KQP) into one pair per complex
// right-hand side (U2c, parts x 2 KQN): |u|^2 = |u_r|^2 + |u_i|^2, the same for dx.  With P null
// only the fold runs (after the correction from the packed tiles).
template <typename T>
__global__ void __launch_bounds__(256)
complex_combine_kernel(const double* __restrict__ P, int nparts, int n, int kc, int KQP,
                       const double* __restrict__ Y, double lambda, double* __restrict__ R, T* __restrict__ Zb,
                       int KQN, int n_pad, const double* __restrict__ U2part, int uparts, double* __restrict__ U2c,
                       const DevStatus* st, int honor_stop) {
    if (block_should_exit(st, honor_stop)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n2 = 2 * (int64_t)n;
    if (P != nullptr && t < (int64_t)n_pad * KQN) {
        const int64_t row = t / KQN;
        const int q = (int)(t % KQN);
        double v = 0.0;
        if (row < n2 && q < kc) {
            const bool im = row >= n;
            const int64_t i = im ? row - n : row;
            // real part: + P[i][q] - P[n+i][kc+q]; imaginary part: + P[n+i][q] + P[i][kc+q]
            const int64_t a = (im ? n + i : i) * KQP + q;
            const int64_t b = (im ? i : n + i) * KQP + kc + q;
            const double sb = im ? 1.0 : -1.0;
            const int64_t stride = n2 * KQP;
            double sa = 0.0, sbb = 0.0;
            for (int p = 0; p < nparts; ++p) {
                sa += P[p * stride + a];
                sbb += P[p * stride + b];
            }
            v = sa + sb * sbb;
            if (Y != nullptr) v -= lambda * Y[row * KQN + q];
        }
        R[t] = v;
        Zb[t] = (T)v;
    }
    if (U2part != nullptr && t < (int64_t)uparts * 2 * KQN) {
        const int64_t p = t / (2 * KQN);
        const int j = (int)(t % (2 * KQN));
        const int which = j / KQN, q = j % KQN;
        double v = 0.0;
        if (q < kc) {
            const double* u = U2part + p * 2 * KQP + which * KQP;
            v = u[q] + u[kc + q];
        }
        U2c[t] = v;
    }
}

// The pass's y columns from the real n-space y (rows 0..2n-1, stride KQN):
//   Yp[row][q] = y_real[row][q],  Yp[row][kc+q] = row < n ? y_real[n+row][q] : -y_real[row-n][q]
// (Z^T of the second column is Im(S^dagger y)); other columns, and rows 2n..rows_out-1, zero.
// FP64 for the passes' y, FP32 for the packed-tile correction's dy.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256)
complex_yexp_kernel(const TI* __restrict__ Y, int KQN, int n, int kc, int KQP, TO* __restrict__ Yp, int rows_out,
                    const DevStatus* st, int honor_stop) {
    if (block_should_exit(st, honor_stop)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n2 = 2 * (int64_t)n;
    if (t >= (int64_t)rows_out * KQP) return;
    const int64_t row = t / KQP;
    const int c = (int)(t % KQP);
    double v = 0.0;
    if (row < n2) {
        if (c < kc) {
            v = (double)Y[row * KQN + c];
        } else if (c < 2 * kc) {
            const int q = c - kc;
            v = row < n ? (double)Y[(row + n) * KQN + q] : -(double)Y[(row - n) * KQN + q];
        }
    }
    Yp[t] = (TO)v;
}

// W_real (lower triangle, n_pad x n_pad, ld) = R(W) from G = Z Z^T (lower, same size, ld), with
// lambda on the diagonal of rows < 2n and the identity on the padding rows:
//   i, j < n        G[i][j] + G[n+i][n+j]
//   n <= i < 2n, j < n   Im W[i-n][j] = G[i][j] - G[n+j][i-n]
//   n <= j <= i < 2n     G[i-n][j-n] + G[i][j]
// Every G entry read is in its lower triangle.
template <typename T>
__global__ void __launch_bounds__(256)
complex_assemble_kernel(const T* __restrict__ G, int64_t ld, int n, int n_pad, double lambda, T* __restrict__ W) {
    const int64_t i = blockIdx.y;
    const int64_t n2 = 2 * (int64_t)n;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= i && j < n_pad;
         j += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (i >= n2) {
            v = (i == j) ? 1.0 : 0.0;
        } else if (i < n) {
            v = (double)G[i * ld + j] + (double)G[(n + i) * ld + n + j];
            if (i == j) v += lambda;
        } else if (j < n) {
            v = (double)G[i * ld + j] - (double)G[(n + j) * ld + (i - n)];
        } else {
            v = (double)G[(i - n) * ld + (j - n)] + (double)G[i * ld + j];
            if (i == j) v += lambda;
        }
        W[i * ld + j] = (T)v;
    }
}

}  // namespace

cudaError_t launch_complex_combine(int f64, const double* P, int nparts, int n, int kc, int KQP, const double* Y,
                                   double lambda, double* R, void* Zb, int KQN, int n_pad, const double* U2part,
                                   int uparts, double* U2c, const DevStatus* st, int honor_stop,
                                   cudaStream_t stream) {
    int64_t total = (int64_t)n_pad * KQN;
    if (U2part != nullptr && (int64_t)uparts * 2 * KQN > total) total = (int64_t)uparts * 2 * KQN;
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (f64)
        complex_combine_kernel<double><<<grid, 256, 0, stream>>>(P, nparts, n, kc, KQP, Y, lambda, R,
                                                                 static_cast<double*>(Zb), KQN, n_pad, U2part,
                                                                 uparts, U2c, st, honor_stop);
    else
        complex_combine_kernel<float><<<grid, 256, 0, stream>>>(P, nparts, n, kc, KQP, Y, lambda, R,
                                                                static_cast<float*>(Zb), KQN, n_pad, U2part,
                                                                uparts, U2c, st, honor_stop);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_complex_yexp(const double* Y, int KQN, int n, int kc, int KQP, double* Yp, const DevStatus* st,
                                int honor_stop, cudaStream_t stream) {
    const int64_t total = 2 * (int64_t)n * KQP;
    complex_yexp_kernel<double, double><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(Y, KQN, n, kc, KQP, Yp,
                                                                                            2 * n, st, honor_stop);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_complex_dyexp(const float* Z, int KQN, int n, int kc, int KQP, float* dy, int rows_out,
                                 const DevStatus* st, int honor_stop, cudaStream_t stream) {
    const int64_t total = (int64_t)rows_out * KQP;
    complex_yexp_kernel<float, float><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(Z, KQN, n, kc, KQP, dy,
                                                                                          rows_out, st, honor_stop);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_complex_assemble(int f64, const void* G, int64_t ld, int n, int n_pad, double lambda, void* W,
                                    cudaStream_t stream) {
    if (n_pad > 65535) return cudaErrorInvalidValue;  // one CTA row per matrix row (gridDim.y)
    const dim3 grid((unsigned)((n_pad + 255) / 256 < 8 ? (n_pad + 255) / 256 : 8), (unsigned)n_pad);
    if (f64)
        complex_assemble_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double*>(G), ld, n, n_pad, lambda,
                                                                  static_cast<double*>(W));
    else
        complex_assemble_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float*>(G), ld, n, n_pad, lambda,
                                                                 static_cast<float*>(W));
    count_launch();
    return cudaGetLastError();
}

}  // namespace dfs
