// ffb_basis.cu -- the steerable principal components themselves (Alg. 2
// step 5 and Sec. V), from the eigenvectors of the last ffb_eig call:
//   radial eigenfunctions  f^{k,l}(xi_j) = sum_q N_{k,q} J_k(R_{k,q} xi_j / c) u^(k)_l(q)   (Eq. sPCArad)
//   eigenimages            g^{k,l}(r, phi) = sum_q u^(k)_l(q) F^{-1}(psi^{k,q})(r, phi)      (Eq. IFT_FB)
// with F^{-1}(psi^{k,q})(r, phi) = 2 c sqrt(pi) (-1)^q i^k R_{k,q} J_k(2 pi c r)
// / ((2 pi c r)^2 - R_{k,q}^2) e^{i k phi}: the phase i^k is the one obtained
// from the inverse-transform convention of Eq. IPFT (the equation as printed
// carries i^{-k}).  Both in float64 on the GPU.
#include <vector>

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
    FFB_PLAN_HERE(p);
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
    FFB_PLAN_HERE(p);
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

// ---------------------------------------------------------------------------
// Rotation-invariant features from the steerable PCA coefficients (the
// bispectrum-like features mentioned in Sec. I):
//   power      |c_{k,l}|^2
//   bispectrum c_{k1,l1} c_{k2,l2} conj(c_{k1+k2,l3})
// with c_{k,l} = sum_q u^(k)_l(q) (a_{k,q} - mean_q [k = 0]) (Eq. sPCAcoeff).
// An in-plane rotation by alpha multiplies c_{k,l} by e^{-ik alpha}, which
// cancels in both; a reflection conjugates every c.
// ---------------------------------------------------------------------------
// c[i][s] for the S distinct components (sk[s], sl[s]); thread per (i, s)
__global__ void k_steer_coef(const float2 *__restrict__ coef, int64_t n, int P, int S, const int *__restrict__ sk,
                             const int *__restrict__ sl, const double *__restrict__ U, const int *__restrict__ pk_,
                             const int *__restrict__ off_, const int *__restrict__ cov_off,
                             const double *__restrict__ mean, float2 *__restrict__ c) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * S) return;
    const int64_t i = t / S;
    const int s = (int)(t - i * S);
    const int k = sk[s], l = sl[s];
    const int p = pk_[k], o = off_[k];
    const double *Uk = U + cov_off[k];
    double re = 0.0, im = 0.0;
    for (int q = 0; q < p; ++q) {
        const float2 a = coef[i * P + o + q];
        const double u = Uk[(size_t)q * p + l];
        re += u * ((k == 0) ? (double)a.x - mean[q] : (double)a.x);
        im += u * ((k == 0) ? 0.0 : (double)a.y);
    }
    c[t] = make_float2((float)re, (float)im);
}

// features of image i: pow[i][t] = |c_{pi[t]}|^2, bis[i][t] = c_a c_b conj(c_c)
__global__ void k_invariants(const float2 *__restrict__ c, int64_t n, int S, int npow, const int *__restrict__ pi,
                             int nbis, const int3 *__restrict__ bi, float *__restrict__ pw, float2 *__restrict__ bs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = npow + nbis;
    if (t >= n * nf) return;
    const int64_t i = t / nf;
    const int f = (int)(t - i * nf);
    const float2 *ci = c + i * S;
    if (f < npow) {
        const float2 v = ci[pi[f]];
        pw[i * npow + f] = v.x * v.x + v.y * v.y;
    } else {
        const int3 b = bi[f - npow];
        const float2 x = ci[b.x], y = ci[b.y], z = ci[b.z];
        const float2 xy = make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
        bs[i * nbis + (f - npow)] = make_float2(xy.x * z.x + xy.y * z.y, xy.y * z.x - xy.x * z.y);
    }
}

extern "C" int ffb_invariants(ffb_plan_t p, const float *d_coef, int64_t n, int npow, const int *h_pairs,
                              float *d_pow, int nbis, const int *h_triples, float *d_bis, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !d_coef || n < 0 || npow < 0 || nbis < 0) return FFB_ERR_ARG;
    if ((npow > 0 && (!h_pairs || !d_pow)) || (nbis > 0 && (!h_triples || !d_bis))) return FFB_ERR_ARG;
    if (!p->eig_ready) return FFB_ERR_STATE;
    if (n == 0 || npow + nbis == 0) return FFB_OK;
    // distinct components, in order of first use
    std::vector<int> sk, sl, pi(npow);
    std::vector<int3> bi(nbis);
    auto comp = [&](int k, int l) -> int {
        if (k < 0 || k > p->k_max || l < 0 || l >= p->p[k]) return -1;
        for (size_t s = 0; s < sk.size(); ++s)
            if (sk[s] == k && sl[s] == l) return (int)s;
        sk.push_back(k);
        sl.push_back(l);
        return (int)sk.size() - 1;
    };
    for (int t = 0; t < npow; ++t)
        if ((pi[t] = comp(h_pairs[2 * t], h_pairs[2 * t + 1])) < 0) return FFB_ERR_ARG;
    for (int t = 0; t < nbis; ++t) {
        const int *q = h_triples + 5 * t;
        const int a = comp(q[0], q[1]), b = comp(q[2], q[3]), c = comp(q[0] + q[2], q[4]);
        if (a < 0 || b < 0 || c < 0) return FFB_ERR_ARG;
        bi[t] = make_int3(a, b, c);
    }
    const int S = (int)sk.size();
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ints = 2 * (size_t)S + npow + 3 * (size_t)nbis;
    char *buf = nullptr;
    const size_t cbytes = sizeof(float2) * (size_t)n * S;
    int e = ffb_check_cuda(cudaMallocAsync((void **)&buf, cbytes + sizeof(int) * ints + 16, s));
    if (e) return e;
    float2 *dc = (float2 *)buf;
    int *di = (int *)(buf + cbytes);
    std::vector<int> hi;
    hi.reserve(ints);
    hi.insert(hi.end(), sk.begin(), sk.end());
    hi.insert(hi.end(), sl.begin(), sl.end());
    hi.insert(hi.end(), pi.begin(), pi.end());
    for (const int3 &b : bi) {
        hi.push_back(b.x);
        hi.push_back(b.y);
        hi.push_back(b.z);
    }
    e = ffb_check_cuda(cudaMemcpyAsync(di, hi.data(), sizeof(int) * ints, cudaMemcpyHostToDevice, s));
    if (!e) {
        const int64_t t1 = n * S, t2 = n * (npow + nbis);
        k_steer_coef<<<(unsigned)((t1 + 255) / 256), 256, 0, s>>>((const float2 *)d_coef, n, p->P, S, di, di + S,
                                                                   p->d_evecs, p->d_p, p->d_off, p->d_cov_off,
                                                                   p->d_mean, dc);
        k_invariants<<<(unsigned)((t2 + 255) / 256), 256, 0, s>>>(dc, n, S, npow, di + 2 * S, nbis,
                                                                  (const int3 *)(di + 2 * S + npow), d_pow,
                                                                  (float2 *)d_bis);
        p->launches += 2;
        e = ffb_check_cuda(cudaGetLastError());
    }
    cudaFreeAsync(buf, s);
    if (e) return e;
    return ffb_check_cuda(cudaStreamSynchronize(s));
}
