// ffb_estimate.cu -- radius of compact support R and band limit c of a stack,
// estimated from the noisy images themselves (the procedure of Sec. V used
// on the simulated ribosome projections):
//   real domain     mean image; per-pixel variance; its mean over rings of
//                   radius r (the mean radial variance); the excess over the
//                   noise variance accumulated with the weight r dr; R is the
//                   radius at which the cumulative fraction reaches `frac`;
//   Fourier domain  the same with the angular average of the mean power
//                   spectrum and the weight xi dxi, giving c.
// Discretisation: rings are the rounded pixel radius r = round(|i|), r < L/2;
// the noise variance, unless given, is the mean variance of the pixels with
// |i| >= L/2 (outside the inscribed disk); the power spectrum is sampled on the
// plan's polar grid (Gauss-Legendre radii, half-plane angles, which suffice
// since |F(-xi)| = |F(xi)| for real images), normalised by L^2 so that white
// noise of variance s^2 gives the level s^2, and integrated with the plan's
// radial quadrature xi_j w_j; the excess over the noise is clipped at zero.
//
// GPU work: one pass of pixel moments (sums of I - s and (I - s)^2 with the
// first image as shift s), the polar transform of the mean image, and per
// chunk the polar transform of the images (the path of ffb_polar) reduced to
// sum_l |F(I) - F(mean)|^2 per radius in float64.
#include <cmath>
#include <vector>

#include "ffb_internal.cuh"

#define CKE(call)                    \
    do {                             \
        int _s = (call);             \
        if (_s != FFB_OK) return _s; \
    } while (0)

// sums over the images [ib, ie) of the CTA's range of (I - s) and (I - s)^2
// per pixel, s = image 0; grid (pixel blocks, image ranges)
__global__ void k_moments(const float *__restrict__ images, int64_t n, int npix, int64_t per,
                          double *__restrict__ sum, double *__restrict__ sq) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npix) return;
    const int64_t ib = (int64_t)blockIdx.y * per;
    const int64_t ie = min(n, ib + per);
    const float s = images[px];
    float a = 0.f, b = 0.f;
    double ad = 0.0, bd = 0.0;
    int cnt = 0;
    for (int64_t i = ib; i < ie; ++i) {
        const float d = images[i * npix + px] - s;
        a += d;
        b = fmaf(d, d, b);
        if (++cnt == 64) {   // float32 partial sums of 64 images, folded into float64
            ad += a;
            bd += b;
            a = b = 0.f;
            cnt = 0;
        }
    }
    atomicAdd(&sum[px], ad + a);
    atomicAdd(&sq[px], bd + b);
}

// mean image (float32, input of the polar transform) and variance map
__global__ void k_moments_final(const float *__restrict__ images, int64_t n, int npix,
                                const double *__restrict__ sum, const double *__restrict__ sq,
                                float *__restrict__ mean, double *__restrict__ var) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npix) return;
    const double d = sum[px] / (double)n;
    mean[px] = (float)((double)images[px] + d);
    var[px] = fmax(sq[px] / (double)n - d * d, 0.0);
}

// pw[j] += sum over the chunk's images and the half-ring angles of
// |F(img, j, l) - Fm(j, l)|^2; grid (n_xi, image groups)
__global__ void k_polar_power(const float2 *__restrict__ F, const float2 *__restrict__ Fm, int m, int n_xi,
                              int nh, int per, double *__restrict__ pw) {
    const int j = blockIdx.x;
    const int i0 = blockIdx.y * per;
    const int i1 = min(m, i0 + per);
    float acc = 0.f;
    for (int i = i0; i < i1; ++i) {
        const float2 *row = F + ((size_t)i * n_xi + j) * nh;
        for (int l = threadIdx.x; l < nh; l += blockDim.x) {
            const float2 a = row[l], b = Fm[(size_t)j * nh + l];
            const float dx = a.x - b.x, dy = a.y - b.y;
            acc = fmaf(dx, dx, fmaf(dy, dy, acc));
        }
    }
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&pw[j], (double)red[0]);
}

static int polar_chunk(ffb_plan_t p, const float *d_images, int64_t i0, int m, float2 *F, cudaStream_t s) {
    if (p->fused) return ffb_launch_fused_polar(p, d_images, i0, m, F, s);
    CKE(ffb_launch_grid(p, d_images, i0, m, s));
    return ffb_launch_polar(p, m, (float *)F, s);
}

// first index at which the running sum of max(v - level, 0) wt reaches frac
// of its total; -1 when the total is zero
static int cut(const std::vector<double> &v, const std::vector<double> &wt, double level, double frac) {
    double tot = 0.0;
    for (size_t i = 0; i < v.size(); ++i) tot += std::max(v[i] - level, 0.0) * wt[i];
    if (!(tot > 0.0)) return -1;
    double run = 0.0;
    for (size_t i = 0; i < v.size(); ++i) {
        run += std::max(v[i] - level, 0.0) * wt[i];
        if (run >= frac * tot) return (int)i;
    }
    return (int)v.size() - 1;
}

extern "C" int ffb_estimate_support(ffb_plan_t p, const float *d_images, int64_t n, double frac, double sigma2,
                                    double *h_out, double *h_radvar, double *h_radpow, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !d_images || !h_out || n < 1 || !(frac > 0.0 && frac <= 1.0)) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->L, npix = L * L, nh = p->n_theta / 2, n_xi = p->n_xi;
    CKE(ffb_ensure_scratch(p));
    // device scratch of this call: moments, mean image, variance map, power,
    // the mean image's polar samples and (separate-kernel path) one chunk's
    const size_t nF = p->fused ? 0 : (size_t)p->chunk * n_xi * nh;
    double *dbuf = nullptr;
    const size_t nd = 3 * (size_t)npix + n_xi;
    const size_t bytes = sizeof(double) * nd + sizeof(float) * npix + sizeof(float2) * ((size_t)n_xi * nh + nF) + 256;
    CKE(ffb_check_cuda(cudaMallocAsync((void **)&dbuf, bytes, s)));
    double *sum = dbuf, *sq = dbuf + npix, *var = dbuf + 2 * npix, *pw = dbuf + 3 * npix;
    float *mean = (float *)(dbuf + nd);
    float2 *Fm = (float2 *)(((uintptr_t)(mean + npix) + 15) & ~(uintptr_t)15);
    float2 *Fc = p->fused ? p->d_Fpol : Fm + (size_t)n_xi * nh;
    int e = ffb_check_cuda(cudaMemsetAsync(dbuf, 0, sizeof(double) * nd, s));
    if (!e) {
        const int64_t per = 1024;
        const int64_t nr = (n + per - 1) / per;
        if (nr > 65535) e = FFB_ERR_ARG;
        if (!e) {
            k_moments<<<dim3((npix + 255) / 256, (unsigned)nr), 256, 0, s>>>(d_images, n, npix, per, sum, sq);
            k_moments_final<<<(npix + 255) / 256, 256, 0, s>>>(d_images, n, npix, sum, sq, mean, var);
            p->launches += 2;
            e = ffb_check_cuda(cudaGetLastError());
        }
    }
    if (!e) e = polar_chunk(p, mean, 0, 1, Fm, s);
    for (int64_t i0 = 0; i0 < n && !e; i0 += p->chunk) {
        const int m = (int)std::min<int64_t>(p->chunk, n - i0);
        e = polar_chunk(p, d_images, i0, m, Fc, s);
        if (!e) {
            const int per = 16;
            k_polar_power<<<dim3(n_xi, (m + per - 1) / per), 256, 0, s>>>(Fc, Fm, m, n_xi, nh, per, pw);
            p->launches++;
            e = ffb_check_cuda(cudaGetLastError());
        }
    }
    std::vector<double> hvar(npix), hpw(n_xi), xi(n_xi), wq(n_xi);
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(hvar.data(), var, sizeof(double) * npix, cudaMemcpyDeviceToHost, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(hpw.data(), pw, sizeof(double) * n_xi, cudaMemcpyDeviceToHost, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(xi.data(), p->d_xi, sizeof(double) * n_xi, cudaMemcpyDeviceToHost, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(wq.data(), p->d_wq, sizeof(double) * n_xi, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(dbuf, s);
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (e) return e;
    int st = 0;
    CKE(ffb_check_cuda(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost)));
    if (st != 0) {
        cudaMemset(p->d_status, 0, sizeof(int));
        return st;
    }
    // rings r = round(|i|) < L/2 and the corners |i| >= L/2, i = a - L/2
    const int nr = L / 2;
    std::vector<double> ring(nr, 0.0), rw(nr);
    std::vector<int64_t> cnt(nr, 0);
    double corner = 0.0;
    int64_t ncorner = 0;
    for (int a1 = 0; a1 < L; ++a1)
        for (int a2 = 0; a2 < L; ++a2) {
            const double x = a1 - L / 2, y = a2 - L / 2;
            const double r = std::sqrt(x * x + y * y);
            const double v = hvar[(size_t)a1 * L + a2];
            const long rb = std::lround(r);
            if (rb < nr) {
                ring[rb] += v;
                cnt[rb]++;
            }
            if (r >= 0.5 * L) {
                corner += v;
                ncorner++;
            }
        }
    for (int r = 0; r < nr; ++r) {
        ring[r] = cnt[r] ? ring[r] / (double)cnt[r] : 0.0;
        rw[r] = (double)r;
    }
    const double s2 = (sigma2 >= 0.0) ? sigma2 : (ncorner ? corner / (double)ncorner : 0.0);
    std::vector<double> pww(n_xi);
    for (int j = 0; j < n_xi; ++j) {
        hpw[j] /= (double)n * (double)nh * (double)L * (double)L;
        pww[j] = xi[j] * wq[j];
    }
    const int iR = cut(ring, rw, s2, frac);
    const int ic = cut(hpw, pww, s2, frac);
    h_out[0] = iR >= 0 ? (double)iR : 0.0;
    h_out[1] = ic >= 0 ? xi[ic] : 0.0;
    h_out[2] = s2;
    h_out[3] = (double)ic;
    if (h_radvar)
        for (int r = 0; r < nr; ++r) h_radvar[r] = ring[r];
    if (h_radpow)
        for (int j = 0; j < n_xi; ++j) h_radpow[j] = hpw[j];
    return FFB_OK;
}
