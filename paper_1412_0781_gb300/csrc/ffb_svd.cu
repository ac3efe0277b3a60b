// ffb_svd.cu -- the SVD route (Sec. III after Eqs. ck, ck_0; Alg. 2 step 4): principal
// components from the coefficient matrices A^(k) directly, without forming the
// covariance from the data.
//
// For each k the real matrix X_k holds one row per image and part: rows
// (Re a_{i,k,.}, Im a_{i,k,.}) for k > 0 (2n rows), rows Re a_{i,0,.} - mean
// for k = 0 (n rows), so that C^(k) = X_k^T X_k / n (Eqs. ck, ck_0).  A
// tall-skinny QR gives X_k = Q_k R_k; the right singular vectors of X_k (the
// left singular vectors of A^(k) in the paper's p_k x n orientation) and its
// singular values s are the eigenvectors and s^2 eigenvalues of R_k^T R_k:
//   * k_tsqr: CTA (k, range) runs an incremental Householder QR over its rows
//     in shared memory (float32 data, float64 norms), each step the running R
//     stacked on the next 256 - p_k rows;
//   * k_tsqr_merge: one CTA per k merges the ranges' R factors pairwise the
//     same way and writes R^T R / n in float64 to the packed block layout;
//   * the batched float64 Jacobi of ffb_eig then returns the eigenpairs (the
//     product R^T R is formed in float64 from the orthogonally reduced R, so no
//     precision is lost to squaring beyond float64 rounding).
#include <algorithm>
#include <vector>

#include "ffb_internal.cuh"

#define TSQR_MB 256       // rows of one QR block
#define TSQR_THREADS 256

// Householder QR of the m x p block X (column-major, leading dimension ld)
// in place; on return the upper triangle of rows 0..p-1 holds R (its
// diagonal may be negative).  One warp per column for the updates.
__device__ void block_qr(float *X, int ld, int m, int p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = TSQR_THREADS / 32;
    __shared__ double red[NW];
    __shared__ float sh_vj, sh_alpha, sh_beta;
    for (int j = 0; j < p && j < m; ++j) {
        float *xj = X + (size_t)j * ld;
        double part = 0.0;
        for (int r = j + 1 + threadIdx.x; r < m; r += TSQR_THREADS) part += (double)xj[r] * xj[r];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tail = 0.0;
            for (int w = 0; w < NW; ++w) tail += red[w];
            const double x0 = xj[j];
            const double nrm = sqrt(x0 * x0 + tail);
            const double alpha = (x0 >= 0.0) ? -nrm : nrm;       // reflect onto -sign(x0) |x| e_j
            const double vj = x0 - alpha;
            const double vtv = vj * vj + tail;
            sh_vj = (float)vj;
            sh_alpha = (float)alpha;
            sh_beta = (vtv > 0.0) ? (float)(2.0 / vtv) : 0.f;
        }
        __syncthreads();
        const float vj = sh_vj, beta = sh_beta;
        if (beta != 0.f) {
            for (int c = j + 1 + warp; c < p; c += NW) {
                float *xc = X + (size_t)c * ld;
                float d = (lane == 0) ? vj * xc[j] : 0.f;
                for (int r = j + 1 + lane; r < m; r += 32) d = fmaf(xj[r], xc[r], d);
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                const float f = beta * d;
                if (lane == 0) xc[j] -= f * vj;
                for (int r = j + 1 + lane; r < m; r += 32) xc[r] = fmaf(-f, xj[r], xc[r]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) xj[j] = (beta != 0.f) ? sh_alpha : xj[j];
        for (int r = j + 1 + threadIdx.x; r < m; r += TSQR_THREADS) xj[r] = 0.f;
        __syncthreads();
    }
}

// value of row rho, column q of X_k
__device__ __forceinline__ float xk(const float2 *coef, int P, int o, int k, const double *mean, int64_t rho, int q) {
    if (k == 0) return (float)((double)coef[rho * P + o + q].x - mean[q]);
    const float2 v = coef[(rho >> 1) * P + o + q];
    return (rho & 1) ? v.y : v.x;
}

// grid (ranges, k_max + 1): R of rows [rb, re) of X_k into Rout[k][range]
// (p_k x p_k, row-major, float32)
__global__ void __launch_bounds__(TSQR_THREADS)
k_tsqr(const float2 *__restrict__ coef, int64_t n, int P, const int *__restrict__ pk_, const int *__restrict__ off_,
       const double *__restrict__ mean, int64_t per, int pmax, float *__restrict__ Rout) {
    extern __shared__ float Xs[];
    const int k = blockIdx.y;
    const int p = pk_[k], o = off_[k];
    const int ld = TSQR_MB + 1;
    const int64_t nrows = (k == 0) ? n : 2 * n;
    const int64_t rb = (int64_t)blockIdx.x * per;
    const int64_t re = min(nrows, rb + per);
    float *Rk = Rout + ((size_t)k * gridDim.x + blockIdx.x) * pmax * pmax;
    int have = 0;   // rows of the running R in the block (0 until the first step)
    for (int64_t r0 = rb; r0 < re || have == 0; ) {
        const int64_t left = (re > r0) ? re - r0 : 0;
        const int take = (int)((left < (int64_t)(TSQR_MB - have)) ? left : (int64_t)(TSQR_MB - have));
        for (int e = threadIdx.x; e < p * (TSQR_MB); e += TSQR_THREADS) {
            const int c = e / TSQR_MB, r = e - c * TSQR_MB;
            if (r >= have) {
                const int64_t rho = r0 + (r - have);
                Xs[(size_t)c * ld + r] = (r - have < take) ? xk(coef, P, o, k, mean, rho, c) : 0.f;
            }
        }
        __syncthreads();
        const int m = max(have + take, p);
        block_qr(Xs, ld, m, p);
        have = p;
        r0 += take;
        if (take == 0) break;
    }
    for (int e = threadIdx.x; e < p * p; e += TSQR_THREADS) {
        const int a = e / p, c = e - a * p;
        Rk[(size_t)a * p + c] = (c >= a) ? Xs[(size_t)c * ld + a] : 0.f;
    }
}

// one CTA per k: merge the ranges' R factors, then C = R^T R / n (float64)
// into the packed block of k
__global__ void __launch_bounds__(TSQR_THREADS)
k_tsqr_merge(const float *__restrict__ Rin, int nranges, const int *__restrict__ pk_, const int *__restrict__ cov_off,
             int pmax, double n, double *__restrict__ C) {
    extern __shared__ float Xs[];
    const int k = blockIdx.x;
    const int p = pk_[k];
    const int ld = TSQR_MB + 1;
    const float *Rk = Rin + (size_t)k * nranges * pmax * pmax;
    const int per_step = max(1, TSQR_MB / p - 1);   // new R factors stacked under the running one
    int have = 0, cnt = 0;
    for (int g = 0; g < nranges; g += cnt) {
        cnt = min(have ? per_step : per_step + 1, nranges - g);   // factors stacked in this step
        for (int e = threadIdx.x; e < p * TSQR_MB; e += TSQR_THREADS) {
            const int c = e / TSQR_MB, r = e - c * TSQR_MB;
            if (r >= have) {
                const int f = (r - have) / p, a = (r - have) - f * p;
                Xs[(size_t)c * ld + r] = (f < cnt) ? Rk[((size_t)(g + f) * pmax * pmax) + (size_t)a * p + c] : 0.f;
            }
        }
        __syncthreads();
        block_qr(Xs, ld, max(have + cnt * p, p), p);
        have = p;
        __syncthreads();
    }
    double *Ck = C + cov_off[k];
    for (int e = threadIdx.x; e < p * p; e += TSQR_THREADS) {
        const int a = e / p, b = e - a * p;
        double s = 0.0;
        for (int r = 0; r <= min(a, b); ++r) s += (double)Xs[(size_t)a * ld + r] * (double)Xs[(size_t)b * ld + r];
        Ck[e] = s / n;
    }
}

// k = 0 mean of Re a_{i,0,q} in float64: block b sums the images
// [512 b, 512 b + 512) (thread: row q = t % 64, every fourth image from
// t / 64) into sum[q] by atomics; k_mean0_final divides by n
#define MEAN0_PER 512
__global__ void __launch_bounds__(256) k_mean0(const float2 *__restrict__ coef, int64_t n, int P, int p0,
                                               double *__restrict__ sum) {
    const int q = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int64_t i0 = (int64_t)blockIdx.x * MEAN0_PER;
    const int64_t i1 = min(n, i0 + MEAN0_PER);
    for (int qq = q; qq < p0; qq += 64) {
        double s = 0.0;
        for (int64_t i = i0 + grp; i < i1; i += 4) s += (double)coef[i * P + qq].x;
        atomicAdd(&sum[qq], s);
    }
}
__global__ void k_mean0_final(int p0, double n, double *__restrict__ mean) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < p0) mean[q] /= n;
}

extern "C" int ffb_svd(ffb_plan_t p, const float *d_coef, int64_t n, double *d_evals, double *d_evecs, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !d_coef || n < 1) return FFB_ERR_ARG;
    if (p->pmax > TSQR_MB / 2) return FFB_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // ranges per k: about sixteen CTAs per SM over all k (each CTA's QR steps
    // run one after another, so shorter ranges shorten the chain), at least
    // 2 p_max rows each
    int64_t nr = (16LL * sms + p->k_max) / (p->k_max + 1);
    nr = std::max<int64_t>(1, std::min<int64_t>(nr, (2 * n) / (2 * p->pmax) + 1));
    const int64_t per0 = (2 * n + nr - 1) / nr;
    const size_t smem = sizeof(float) * (size_t)p->pmax * (TSQR_MB + 1);
    static int attr = 0;
    if (attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_tsqr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (!e) e = ffb_check_cuda(cudaFuncSetAttribute(k_tsqr_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    float *R = nullptr;
    const size_t nR = (size_t)(p->k_max + 1) * nr * p->pmax * p->pmax;
    int e = ffb_check_cuda(cudaMallocAsync((void **)&R, sizeof(float) * nR, s));
    if (e) return e;
    {
        ProfScope ps(p, FFB_KC_EIG, s);
        e = ffb_check_cuda(cudaMemsetAsync(p->d_mean, 0, sizeof(double) * p->p[0], s));
        k_mean0<<<(unsigned)((n + MEAN0_PER - 1) / MEAN0_PER), 256, 0, s>>>((const float2 *)d_coef, n, p->P, p->p[0],
                                                                        p->d_mean);
        k_mean0_final<<<(p->p[0] + 63) / 64, 64, 0, s>>>(p->p[0], (double)n, p->d_mean);
        // k = 0 has n rows, k > 0 have 2n: the k = 0 ranges use half the length
        k_tsqr<<<dim3((unsigned)nr, p->k_max + 1), TSQR_THREADS, smem, s>>>(
            (const float2 *)d_coef, n, p->P, p->d_p, p->d_off, p->d_mean, per0, p->pmax, R);
        k_tsqr_merge<<<p->k_max + 1, TSQR_THREADS, smem, s>>>(R, (int)nr, p->d_p, p->d_cov_off, p->pmax, (double)n,
                                                               p->d_Cfin);
        p->launches += 4;
        e = ffb_check_cuda(cudaGetLastError());
    }
    cudaFreeAsync(R, s);
    if (e) return e;
    e = ffb_launch_eig(p, s);
    if (e) return e;
    p->eig_ready = 1;
    if (d_evals)
        e = ffb_check_cuda(cudaMemcpyAsync(d_evals, p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, s));
    if (!e && d_evecs)
        e = ffb_check_cuda(
            cudaMemcpyAsync(d_evecs, p->d_evecs, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s));
    if (e) return e;
    return ffb_sync(p, stream);
}
