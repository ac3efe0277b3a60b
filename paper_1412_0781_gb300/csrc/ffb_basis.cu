// ffb_basis.cu -- the steerable principal components themselves (Alg. 2
// step 5 and Sec. V), from the eigenvectors of the last ffb_eig call:
//   radial eigenfunctions  f^{k,l}(xi_j) = sum_q N_{k,q} J_k(R_{k,q} xi_j / c) u^(k)_l(q)   (Eq. sPCArad)
//   eigenimages            g^{k,l}(r, phi) = sum_q u^(k)_l(q) F^{-1}(psi^{k,q})(r, phi)      (Eq. IFT_FB)
// with F^{-1}(psi^{k,q})(r, phi) = 2 c sqrt(pi) (-1)^q i^k R_{k,q} J_k(2 pi c r)
// / ((2 pi c r)^2 - R_{k,q}^2) e^{i k phi}: the phase i^k is the one obtained
// from the inverse-transform convention of Eq. IPFT (the equation as printed
// carries i^{-k}).  Both in float64 on the GPU.
#include "ffb_internal.cuh"

// one CTA per k: f[offset_k * n_xi + j * p_k + l]
__global__ void k_radial_eigfun(const double *__restrict__ B64, const double *__restrict__ xi,
                                const double *__restrict__ wq, const double *__restrict__ U,
                                const int *__restrict__ pk_, const int *__restrict__ off_,
                                const int *__restrict__ cov_off, int n_xi, double *__restrict__ f) {
    const int k = blockIdx.x;
    const int p = pk_[k], o = off_[k];
    const double *Uk = U + cov_off[k];
    for (int e = threadIdx.x; e < n_xi * p; e += blockDim.x) {
        const int j = e / p, l = e % p;
        const double sw = xi[j] * wq[j];
        double s = 0.0;
        for (int q = 0; q < p; ++q) s += B64[(size_t)(o + q) * n_xi + j] / sw * Uk[q * p + l];
        f[(size_t)o * n_xi + e] = s;
    }
}

// one thread per (pair, pixel): out[pair][a1][a2][re, im]
__global__ void k_eigenimages(int npairs, const int *__restrict__ pk_list, const int *__restrict__ pl_list,
                              const double *__restrict__ zeros, const double *__restrict__ U,
                              const int *__restrict__ pk_, const int *__restrict__ off_,
                              const int *__restrict__ cov_off, int L, int off, double c,
                              double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)npairs * L * L) return;
    const int pair = (int)(t / ((int64_t)L * L));
    const int pix = (int)(t % ((int64_t)L * L));
    const int k = pk_list[pair], l = pl_list[pair];
    const int p = pk_[k], o = off_[k];
    const double *Uk = U + cov_off[k];
    const double x1 = (double)(pix / L - off), x2 = (double)(pix % L - off);
    const double r = sqrt(x1 * x1 + x2 * x2);
    const double phi = atan2(x2, x1);
    const double pi = 3.14159265358979323846;
    const double z = 2.0 * pi * c * r;
    const double Jk = bessel_j_miller(k, z);
    double radial = 0.0;
    for (int q = 0; q < p; ++q) {
        const double R = zeros[o + q];
        const double sgn = ((q + 1) & 1) ? -1.0 : 1.0;   // (-1)^q with q 1-based
        double ratio;
        if (fabs(z - R) < 1e-9 * R) ratio = -0.5 * bessel_j_miller(k + 1, R);   // removable point
        else ratio = R * Jk / ((z - R) * (z + R));
        radial += Uk[q * p + l] * sgn * ratio;
    }
    radial *= 2.0 * c * sqrt(pi);
    // i^k e^{i k phi} = e^{i k (phi + pi/2)}
    double sn, cs;
    sincos((double)k * (phi + 0.5 * pi), &sn, &cs);
    out[2 * t] = radial * cs;
    out[2 * t + 1] = radial * sn;
}

extern "C" int ffb_radial_eigenfunctions(ffb_plan_t p, double *d_f, void *stream) {
    if (!p || !d_f) return FFB_ERR_ARG;
    if (!p->eig_ready) return FFB_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    k_radial_eigfun<<<p->k_max + 1, 256, 0, s>>>(p->d_B64, p->d_xi, p->d_wq, p->d_evecs, p->d_p, p->d_off,
                                                 p->d_cov_off, p->n_xi, d_f);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

extern "C" int ffb_eigenimages(ffb_plan_t p, int npairs, const int *h_k, const int *h_l, double *d_out,
                               void *stream) {
    if (!p || npairs < 0 || (npairs > 0 && (!h_k || !h_l || !d_out))) return FFB_ERR_ARG;
    if (!p->eig_ready) return FFB_ERR_STATE;
    if (npairs == 0) return FFB_OK;
    for (int i = 0; i < npairs; ++i)
        if (h_k[i] < 0 || h_k[i] > p->k_max || h_l[i] < 0 || h_l[i] >= p->p[h_k[i]]) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_kl = nullptr;
    int e = ffb_check_cuda(cudaMallocAsync((void **)&d_kl, sizeof(int) * 2 * (size_t)npairs, s));
    if (e) return e;
    e = ffb_check_cuda(cudaMemcpyAsync(d_kl, h_k, sizeof(int) * npairs, cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(d_kl + npairs, h_l, sizeof(int) * npairs, cudaMemcpyHostToDevice, s));
    if (!e) {
        const int64_t tot = (int64_t)npairs * p->L * p->L;
        k_eigenimages<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(npairs, d_kl, d_kl + npairs, p->d_zeros,
                                                                    p->d_evecs, p->d_p, p->d_off, p->d_cov_off,
                                                                    p->L, p->off, p->c, d_out);
        p->launches++;
        e = ffb_check_cuda(cudaGetLastError());
    }
    cudaFreeAsync(d_kl, s);
    if (e) return e;
    return ffb_check_cuda(cudaStreamSynchronize(s));
}
