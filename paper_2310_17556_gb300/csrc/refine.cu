// Device-side control of the n-space iterative refinement (mixed-precision paths).
//
// Algorithm 1 solves the n x n system (S S^T + lambda I~) y = S v (Appendix A) with the factor
// of W = S S^T + lambda I~.  When W is formed in low precision (W~ = W + E), y_0 = W~^{-1} S v
// is refined with the exact operator:  r = S v - (S S^T + lambda I~) y = S (v - S^T y) - lambda y
// (one pass over S, pass.cu), dy = W~^{-1} r (trsv.cu), y += dy.  The x of Algorithm 1's update,
// x_j = (v - S^T y_j) / lambda, is written by the same pass, which also measures exactly how
// much x moved:  delta_j = ||x_j - x_{j-1}|| / ||x_j||  (x_0 = v / lambda, i.e. y = 0).
// With linear convergence at rate rho_j = delta_j / delta_{j-1}, the error left in x_j is about
// delta_j rho_j / (1 - rho_j).  Stop (converged) once that estimate is <= tol; stop with
// NOT_CONVERGED when the iteration budget is used up or rho_j >= 0.9 (stagnation, e.g. at the
// rounding floor of the passes, or divergence).  Once stopped, every later kernel of the solve
// sees `stop` and returns at once, so a fixed launch sequence serves any iteration count with no
// host round trip.
#include "kernels.cuh"

namespace dfs {

__global__ void status_reset_kernel(DevStatus* st, unsigned long long wait_ns, int fault) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->status = 0;
        st->failed_pivot = -1;
        st->converged = 0;
        st->iters = 0;
        st->stop = 0;
        st->passes = 0;
        st->rel_correction = 0.0;
        st->rel_residual = 0.0;
        st->prev_correction = 0.0;
        st->wait_ns = wait_ns;
        st->fault = fault;
        st->bounds_site = 0;
    }
}

// After the first solve: y = z (the solve type T -> FP64), remember ||b|| per RHS.
template <typename T>
__global__ void __launch_bounds__(256)
refine_init_kernel(const T* __restrict__ Z, int n_pad, int KQ, double* __restrict__ Y,
                   const double* __restrict__ R, double* __restrict__ bnorm2, DevStatus* st) {
    if (block_should_exit(st, 0)) return;
    __shared__ double red[8][8];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < n_pad * KQ; e += blockDim.x) {
        Y[e] = (double)Z[e];
        const double r = R[e];
        acc[e % KQ] += r * r;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = 0; q < 8; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < KQ) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        bnorm2[threadIdx.x] = v;
    }
}

// After pass `it` of the refinement (or the correction from the packed tiles): sum the passes'
// per-part statistics into U2 (sum u^2 = lambda^2 ||x||^2, sum (x_new - x_old)^2, per RHS), form
// delta_it and the rate, and decide.  `fast`: x came from the packed BF16 tiles, whose rounding
// (2^-9 relative, of a correction of relative size delta) adds up to 2^-8 delta to the error
// estimate; if that run does not converge, nothing else is decided here (the full pass that
// follows recomputes x exactly and the next check carries on from delta_it).
__global__ void __launch_bounds__(512)
refine_check_kernel(const double* __restrict__ U2part, int nparts, double* __restrict__ U2, int KQ, int k,
                    double lambda, double tol, int it, int max_iter, int fast, DevStatus* st) {
    if (block_should_exit(st, 1)) return;
    __shared__ double u2[16];
    // one warp per statistic: lanes take the parts lane, lane + 32, ..., then a fixed shuffle tree
    // (a fixed summation order, so the result does not vary run to run)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2 * KQ) {
        double u = 0.0;
        for (int b = lane; b < nparts; b += 32) u += U2part[(int64_t)b * 2 * KQ + warp];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (lane == 0) {
            u2[warp] = u;
            U2[warp] = u;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double delta = 0.0;
    bool finite = true;
    for (int q = 0; q < k && q < KQ; ++q) {
        // ||x_j - x_{j-1}|| / ||x_j|| with ||x_j|| = ||u|| / lambda
        const double dq = lambda * sqrt(u2[KQ + q]) / fmax(sqrt(u2[q]), 1e-300);
        if (!isfinite(dq)) finite = false;
        delta = fmax(delta, dq);
    }
    const double prev = st->prev_correction;
    double est = delta;
    bool have_rate = false;
    double rho = 0.0;
    if (it > 1 && prev > 0.0) {
        rho = delta / prev;
        have_rate = true;
        est = delta * rho / (1.0 - fmin(rho, 0.99));
    }
    if (fast) est += delta * (1.0 / 256.0);
    st->rel_correction = est;
    st->iters = it;
    st->prev_correction = delta;
    if (!finite) {
        set_status(st, DFS_ERR_NONFINITE);
        st->stop = 1;
    } else if ((have_rate && est <= tol) || (!fast && delta <= 1e-2 * tol)) {
        st->converged = 1;
        st->stop = 1;
        st->passes = fast ? it - 1 : it;
    } else if (!fast && (it >= max_iter || (have_rate && rho >= 0.9))) {
        set_status(st, DFS_ERR_NOT_CONVERGED);
        st->stop = 1;
        st->passes = it;
    }
}

// After the n-space solve of a refinement step that did not stop: y += dy, and the relative
// n-space residual ||r|| / ||b|| of that step (reported in dfs_info).
template <typename T>
__global__ void __launch_bounds__(256)
refine_update_kernel(const T* __restrict__ Z, const double* __restrict__ R, int n_pad, int KQ, int k,
                     double* __restrict__ Y, const double* __restrict__ bnorm2, DevStatus* st) {
    if (block_should_exit(st, 1)) return;
    __shared__ double red[8][8];
    double rr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < n_pad * KQ; e += blockDim.x) {
        const double r = R[e];
        rr[e % KQ] += r * r;
        Y[e] += (double)Z[e];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = 0; q < 8; ++q) {
        double c = rr[q];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) red[warp][q] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double relr = 0.0;
        for (int q = 0; q < k && q < KQ; ++q) {
            double c = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += red[w][q];
            relr = fmax(relr, sqrt(c / fmax(bnorm2[q], 1e-300)));
        }
        st->rel_residual = relr;
    }
}

cudaError_t launch_status_reset(DevStatus* st, cudaStream_t stream, unsigned long long wait_ns, int fault) {
    {
        status_reset_kernel<<<1, 32, 0, stream>>>(st, wait_ns ? wait_ns : kDefaultWaitNs, fault);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_refine_init(int f64, const void* Z, int n_pad, int KQ, double* Y, const double* R,
                               double* bnorm2, DevStatus* st, cudaStream_t stream) {
    if (f64)
        {
            refine_init_kernel<double><<<1, 256, 0, stream>>>(static_cast<const double*>(Z), n_pad, KQ, Y, R, bnorm2, st);
            count_launch();
        }
    else
        {
            refine_init_kernel<float><<<1, 256, 0, stream>>>(static_cast<const float*>(Z), n_pad, KQ, Y, R, bnorm2, st);
            count_launch();
        }
    return cudaGetLastError();
}

cudaError_t launch_refine_check(const double* U2part, int nparts, double* U2, int KQ, int k, double lambda, double tol,
                                int it, int max_iter, int fast, DevStatus* st, cudaStream_t stream) {
    if (KQ > 8) return cudaErrorInvalidValue;
    refine_check_kernel<<<1, 64 * KQ, 0, stream>>>(U2part, nparts, U2, KQ, k, lambda, tol, it, max_iter, fast, st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_refine_update(int f64, const void* Z, const double* R, int n_pad, int KQ, int k, double* Y,
                                 const double* bnorm2, DevStatus* st, cudaStream_t stream) {
    if (f64)
        refine_update_kernel<double><<<1, 256, 0, stream>>>(static_cast<const double*>(Z), R, n_pad, KQ, k, Y, bnorm2, st);
    else
        refine_update_kernel<float><<<1, 256, 0, stream>>>(static_cast<const float*>(Z), R, n_pad, KQ, k, Y, bnorm2, st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dfs
