// ffb_api.cu -- C ABI entry points of the hot path (see include/ffb.h).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ffb_internal.cuh"

#define CK(call)                         \
    do {                                 \
        int _s = (call);                 \
        if (_s != FFB_OK) return _s;     \
    } while (0)

static int read_status(ffb_plan_t p, cudaStream_t s) {
    int st = 0;
    int e = ffb_check_cuda(cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (e) return e;
    e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (e) return e;
    if (st != 0) cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
    return st;
}

extern "C" int ffb_sync(ffb_plan_t p, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p) return FFB_ERR_ARG;
    return read_status(p, (cudaStream_t)stream);
}

extern "C" int ffb_profile(ffb_plan_t p, int enable) {
    if (!p || enable < 0) return FFB_ERR_ARG;
    p->prof_on = enable;
    p->prof_used = 0;
    for (int c = 0; c < 16; ++c) p->prof_calls[c] = 0;
    return FFB_OK;
}

extern "C" int ffb_profile_read(ffb_plan_t p, double *h_ms, int64_t *h_calls) {
    FFB_PLAN_HERE(p);
    if (!p || !h_ms || !h_calls) return FFB_ERR_ARG;
    for (int c = 0; c < FFB_NKC; ++c) {
        h_ms[c] = 0.0;
        h_calls[c] = 0;
    }
    int64_t timed[FFB_NKC] = {};
    for (size_t i = 0; i < p->prof_used; ++i) {
        const ProfEv &e = p->prof[i];
        if (cudaEventSynchronize(e.b) != cudaSuccess) return FFB_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) != cudaSuccess) return FFB_ERR_CUDA;
        h_ms[e.cls] += ms;
        timed[e.cls] += 1;
    }
    // sampled classes: the mean timed duration times the launches
    for (int c = 0; c < FFB_NKC; ++c) {
        h_calls[c] = p->prof_calls[c];
        if (timed[c] > 0) h_ms[c] *= (double)p->prof_calls[c] / (double)timed[c];
        p->prof_calls[c] = 0;
    }
    p->prof_used = 0;
    return FFB_OK;
}

extern "C" int ffb_polar(ffb_plan_t p, const float *d_images, int64_t n, float *d_F, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_images || !d_F))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(ffb_ensure_scratch(p));
    const size_t per = (size_t)p->n_xi * (p->n_theta / 2) * 2;
    for (int64_t i0 = 0; i0 < n; i0 += p->chunk) {
        int m = (int)std::min<int64_t>(p->chunk, n - i0);
        if (p->fused) {
            CK(ffb_launch_fused_polar(p, d_images, i0, m, (float2 *)(d_F + (size_t)i0 * per), s, i0 > 0,
                                      n - (i0 + m)));
        } else {
            CK(ffb_launch_grid(p, d_images, i0, m, s));
            CK(ffb_launch_polar(p, m, d_F + (size_t)i0 * per, s));
        }
    }
    return FFB_OK;
}

// a1-a5 launches for n images on stream s (arguments already validated)
// a1-a4 of the images [g0, g1), one group of at most ffb_tc_group chunks,
// into the operands of the radial quadrature (the tensor-core planes, or the
// float32 spectra of the FP32 path)
int ffb_expand_part(ffb_plan_t p, const float *d_images, int64_t g0, int64_t g1, cudaStream_t s) {
    RingOut ring{FFB_FMT_F32, p->d_Fhat, nullptr, p->n_xi, p->chunk};
    if (p->precision != FFB_FP32) CK(ffb_tc_prepare(p, s, &ring));
    const size_t es = (ring.fmt == FFB_FMT_BF16 || ring.fmt == FFB_FMT_BF16X2) ? 2 : 4;
    for (int64_t i0 = g0; i0 < g1; i0 += p->chunk) {
        int m = (int)std::min<int64_t>(p->chunk, g1 - i0);
        if (p->fused) {
            // chunks after the first follow this call's own kernels; where the
            // plan takes the tensor-core ring DFT the grid kernel leaves bf16
            // planes for it
            const bool tcdft = ffb_tc_dft_ok(p);
            CK(ffb_launch_fused_polar(p, d_images, i0, m, p->d_Fpol, s, i0 > 0, g1 - (i0 + m), tcdft));
            RingOut r = ring;   // this chunk's images in the group's planes
            const size_t off = (size_t)(i0 - g0) * 2 * ring.ld * es;
            r.p0 = (char *)ring.p0 + off;
            if (ring.p1) r.p1 = (char *)ring.p1 + off;
            if (tcdft) CK(ffb_launch_tc_dft(p, m, r, s));
            else CK(ffb_launch_ring_fft(p, m, p->d_Fpol, r, s));
        } else if (p->ring_direct) {
            // tiled interpolation into the polar buffer, then the register
            // ring FFT straight into this chunk's quadrature operands
            CK(ffb_launch_grid(p, d_images, i0, m, s));
            CK(ffb_launch_tile_polar(p, m, p->d_Fpol, s));
            RingOut r = ring;
            const size_t off = (size_t)(i0 - g0) * 2 * ring.ld * es;
            r.p0 = (char *)ring.p0 + off;
            if (ring.p1) r.p1 = (char *)ring.p1 + off;
            CK(ffb_launch_ring_fft(p, m, p->d_Fpol, r, s));
        } else {
            CK(ffb_launch_grid(p, d_images, i0, m, s));
            CK(ffb_launch_interp_ring(p, m, s));
        }
    }
    return FFB_OK;
}

int ffb_expand_on(ffb_plan_t p, const float *d_images, int64_t n, float *d_coef, cudaStream_t s) {
    if (n == 0) return FFB_OK;
    CK(ffb_ensure_scratch(p));
    int grp = 1;
    if (p->precision != FFB_FP32) {
        CK(ffb_tc_prepare(p, s, nullptr));
        grp = ffb_tc_group(p);
    }
    // groups of grp chunks: polar transform and ring DFT per chunk, one
    // quadrature launch per group
    for (int64_t g0 = 0; g0 < n; g0 += (int64_t)grp * p->chunk) {
        const int64_t g1 = std::min<int64_t>(n, g0 + (int64_t)grp * p->chunk);
        CK(ffb_expand_part(p, d_images, g0, g1, s));
        CK(ffb_launch_bessel(p, (int)(g1 - g0), d_coef + (size_t)g0 * p->P * 2, p->ring_direct != 0, s));
    }
    return FFB_OK;
}

extern "C" int ffb_expand(ffb_plan_t p, const float *d_images, int64_t n, float *d_coef, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_images || !d_coef))) return FFB_ERR_ARG;
    return ffb_expand_on(p, d_images, n, d_coef, (cudaStream_t)stream);
}

extern "C" int ffb_covariance(ffb_plan_t p, const float *d_coef, int64_t n, int reset, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && !d_coef)) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (reset) {
        CK(ffb_check_cuda(cudaMemsetAsync(p->d_acc, 0, sizeof(double) * p->cov_total, s)));
        CK(ffb_check_cuda(cudaMemsetAsync(p->d_sum0, 0, sizeof(double) * p->p[0], s)));
        p->n_acc = 0;
        p->shift_set = 0;
    }
    if (n == 0) return FFB_OK;
    if (!p->shift_set) {
        CK(ffb_launch_cov_shift(p, d_coef, n, s));
        p->shift_set = 1;
    }
    CK(ffb_launch_cov(p, d_coef, n, s));
    p->n_acc += n;
    return FFB_OK;
}

extern "C" int ffb_cov_get(ffb_plan_t p, double *d_mean0, double *d_C, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    CK(ffb_launch_cov_final(p, s));
    if (d_mean0)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_mean0, p->d_mean, sizeof(double) * p->p[0], cudaMemcpyDeviceToDevice, s)));
    if (d_C)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_C, p->d_Cfin, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    return read_status(p, s);
}

// Images in host memory, statistics back in host memory: the images go to
// the device in parts of host_cap images through a ring of FFB_HOST_SLOTS
// device buffers, copied on the plan's own stream while the previous parts
// are expanded on the caller's; each copy waits only for its slot's previous
// expansion, each expansion only for its own copy.
extern "C" int ffb_expand_cov_host(ffb_plan_t p, const float *h_images, int64_t n, int reset, double *h_mean0,
                                   double *h_C, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && !h_images)) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        CK(ffb_ensure_scratch(p));
        const size_t img_bytes = sizeof(float) * (size_t)p->L * p->L;
        // a part of two quadrature groups, or fewer images where that would
        // exceed 256 MiB per slot (whole chunks, at least one)
        const int64_t grp = (int64_t)(p->precision != FFB_FP32 ? ffb_tc_group(p) : 1) * p->chunk;
        int64_t cap = 2 * grp;
        const int64_t lim = std::max<int64_t>(p->chunk, ((int64_t)(256u << 20) / (int64_t)img_bytes) / p->chunk * p->chunk);
        cap = std::min(cap, lim);
        if (p->host_cap < cap) {
            if (p->h2d) CK(ffb_check_cuda(cudaStreamSynchronize(p->h2d)));
            CK(ffb_check_cuda(cudaStreamSynchronize(s)));
            if (p->d_hostimg) cudaFree(p->d_hostimg);
            if (p->d_hostcoef) cudaFree(p->d_hostcoef);
            p->d_hostimg = nullptr;
            p->d_hostcoef = nullptr;
            p->host_cap = 0;
            CK(ffb_check_cuda(cudaMalloc((void **)&p->d_hostimg, img_bytes * (size_t)cap * FFB_HOST_SLOTS)));
            CK(ffb_check_cuda(cudaMalloc((void **)&p->d_hostcoef, sizeof(float2) * (size_t)cap * p->P)));
            p->host_cap = cap;
        }
        cap = p->host_cap;
        if (!p->h2d) {
            CK(ffb_check_cuda(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking)));
            for (int i = 0; i < FFB_HOST_SLOTS; ++i) {
                CK(ffb_check_cuda(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming)));
                CK(ffb_check_cuda(cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming)));
            }
        }
        // the slots' earlier contents may still be read by work the caller
        // queued on s before this call
        CK(ffb_check_cuda(cudaEventRecord(p->ev_free[0], s)));
        CK(ffb_check_cuda(cudaStreamWaitEvent(p->h2d, p->ev_free[0], 0)));
        int64_t part = 0;
        for (int64_t i0 = 0; i0 < n; i0 += cap, ++part) {
            const int64_t m = std::min(cap, n - i0);
            const int slot = (int)(part % FFB_HOST_SLOTS);
            float *d_img = p->d_hostimg + (size_t)slot * cap * p->L * p->L;
            if (part >= FFB_HOST_SLOTS) CK(ffb_check_cuda(cudaStreamWaitEvent(p->h2d, p->ev_free[slot], 0)));
            CK(ffb_check_cuda(cudaMemcpyAsync(d_img, h_images + (size_t)i0 * p->L * p->L, img_bytes * (size_t)m,
                                              cudaMemcpyHostToDevice, p->h2d)));
            CK(ffb_check_cuda(cudaEventRecord(p->ev_copied[slot], p->h2d)));
            CK(ffb_check_cuda(cudaStreamWaitEvent(s, p->ev_copied[slot], 0)));
            CK(ffb_expand_on(p, d_img, m, p->d_hostcoef, s));
            CK(ffb_check_cuda(cudaEventRecord(p->ev_free[slot], s)));
            CK(ffb_covariance(p, p->d_hostcoef, m, reset && i0 == 0, stream));
        }
    } else if (reset) {
        CK(ffb_covariance(p, nullptr, 0, 1, stream));
    }
    if (!h_mean0 && !h_C) return read_status(p, s);
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    CK(ffb_launch_cov_final(p, s));
    if (h_mean0)
        CK(ffb_check_cuda(cudaMemcpyAsync(h_mean0, p->d_mean, sizeof(double) * p->p[0], cudaMemcpyDeviceToHost, s)));
    if (h_C)
        CK(ffb_check_cuda(cudaMemcpyAsync(h_C, p->d_Cfin, sizeof(double) * p->cov_total, cudaMemcpyDeviceToHost, s)));
    return read_status(p, s);
}

extern "C" int ffb_eig(ffb_plan_t p, double *d_evals, double *d_evecs, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    CK(ffb_launch_cov_final(p, s));
    CK(ffb_launch_eig(p, s));
    p->eig_ready = 1;
    if (d_evals)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evals, p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, s)));
    if (d_evecs)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evecs, p->d_evecs, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    return read_status(p, s);
}

extern "C" int ffb_eig_blocks(ffb_plan_t p, const double *d_C, double *d_evals, double *d_evecs, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !d_C) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_Cfin, d_C, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    CK(ffb_launch_eig(p, s));
    p->eig_ready = 1;
    if (d_evals)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evals, p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, s)));
    if (d_evecs)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evecs, p->d_evecs, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    return read_status(p, s);
}

extern "C" int ffb_expand_adjoint(ffb_plan_t p, const float *d_coef, int64_t n, float *d_images, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_coef || !d_images))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    return ffb_launch_adjoint(p, d_coef, n, d_images, (cudaStream_t)stream);
}

// Selection of the steerable components (Sec. V), host side: gains h for
// every (k, l) from the per-block descending eigenvalues.
static void select_gains(ffb_plan_t p, const std::vector<double> &ev, int mode, int K, double sigma2, int64_t n,
                         std::vector<double> &h) {
    h.assign(p->P, 0.0);
    if (mode == FFB_DENOISE_ALL) {
        h.assign(p->P, 1.0);
        return;
    }
    if (mode == FFB_DENOISE_TOPK) {
        // rank pairs (k, l) by eigenvalue, ties by smaller k then smaller l
        std::vector<int> idx(p->P);
        std::vector<int> kof(p->P);
        for (int k = 0; k <= p->k_max; ++k)
            for (int l = 0; l < p->p[k]; ++l) kof[p->offset[k] + l] = k;
        for (int i = 0; i < p->P; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            if (ev[a] != ev[b]) return ev[a] > ev[b];
            if (kof[a] != kof[b]) return kof[a] < kof[b];
            return a < b;
        });
        for (int i = 0; i < K && i < p->P; ++i) h[idx[i]] = 1.0;
        return;
    }
    // Marchenko-Pastur edge (Eq. compselect); gain (lambda - sigma2)/lambda
    // (Wiener form of the soft threshold) or 1 (hard selection)
    for (int k = 0; k <= p->k_max; ++k) {
        double gamma = (k == 0) ? (double)p->p[k] / (double)n : (double)p->p[k] / (2.0 * (double)n);
        double thr = sigma2 * (1.0 + std::sqrt(gamma)) * (1.0 + std::sqrt(gamma));
        for (int l = 0; l < p->p[k]; ++l) {
            double lam = ev[p->offset[k] + l];
            if (lam > thr) h[p->offset[k] + l] = (mode == FFB_DENOISE_MP_HARD) ? 1.0 : (lam - sigma2) / lam;
        }
    }
}

extern "C" int ffb_select(ffb_plan_t p, int mode, int K, double sigma2, int64_t n, double *h_gain, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p) return FFB_ERR_ARG;
    if (mode < FFB_DENOISE_TOPK || mode > FFB_DENOISE_MP_HARD) return FFB_ERR_ARG;
    if (mode == FFB_DENOISE_TOPK && K < 0) return FFB_ERR_ARG;
    if ((mode == FFB_DENOISE_MP_WIENER || mode == FFB_DENOISE_MP_HARD) && (!(sigma2 >= 0.0) || n <= 0))
        return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->d_gain) CK(ffb_check_cuda(cudaMalloc(&p->d_gain, sizeof(double) * p->P)));
    if (!p->d_M) CK(ffb_check_cuda(cudaMalloc(&p->d_M, sizeof(float) * p->cov_total)));
    std::vector<double> ev(p->P);
    CK(ffb_check_cuda(cudaMemcpyAsync(ev.data(), p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToHost, s)));
    CK(read_status(p, s));
    std::vector<double> h;
    select_gains(p, ev, mode, K, sigma2, n, h);
    if (h_gain) std::copy(h.begin(), h.end(), h_gain);
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_gain, h.data(), sizeof(double) * p->P, cudaMemcpyHostToDevice, s)));
    CK(ffb_launch_filter_matrix(p, s));
    p->selected = 1;
    return read_status(p, s);
}

extern "C" int ffb_filter(ffb_plan_t p, const float *d_coef_in, int64_t n, float *d_coef_out, int flags, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_coef_in || !d_coef_out)) || (flags & ~3)) return FFB_ERR_ARG;
    if (!p->selected) return FFB_ERR_STATE;
    if (n == 0) return FFB_OK;
    return ffb_launch_filter(p, d_coef_in, n, d_coef_out, flags, (cudaStream_t)stream);
}

extern "C" int ffb_weight(ffb_plan_t p, const float *d_coef_in, int64_t n, float *d_coef_out, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_coef_in || !d_coef_out))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    return ffb_launch_weight(p, d_coef_in, n, d_coef_out, (cudaStream_t)stream);
}

extern "C" int ffb_denoise(ffb_plan_t p, const float *d_images, int64_t n, int mode, int K, double sigma2,
                           float *d_out, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n <= 0 || !d_images || !d_out) return FFB_ERR_ARG;
    if (mode < FFB_DENOISE_TOPK || mode > FFB_DENOISE_MP_HARD) return FFB_ERR_ARG;
    if (mode == FFB_DENOISE_TOPK && K < 0) return FFB_ERR_ARG;
    if ((mode == FFB_DENOISE_MP_WIENER || mode == FFB_DENOISE_MP_HARD) && !(sigma2 >= 0.0)) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->den_cap < n) {
        if (p->d_coef_den) cudaFree(p->d_coef_den);
        p->d_coef_den = nullptr;
        p->den_cap = 0;
        CK(ffb_check_cuda(cudaMalloc(&p->d_coef_den, sizeof(float2) * (size_t)n * p->P)));
        p->den_cap = n;
    }
    float *coef = (float *)p->d_coef_den;
    CK(ffb_expand(p, d_images, n, coef, stream));
    CK(ffb_covariance(p, coef, n, 1, stream));
    CK(ffb_launch_cov_final(p, s));
    CK(ffb_launch_eig(p, s));
    p->eig_ready = 1;
    CK(ffb_select(p, mode, K, sigma2, n, nullptr, stream));
    CK(ffb_launch_filter(p, coef, n, coef, FFB_FILTER_WEIGHT, s));
    CK(ffb_launch_adjoint(p, coef, n, d_out, s));
    return read_status(p, s);
}

// ---------------------------------------------------------------------------
// Covariance statistics across processes (images split over GPUs, Sec. IV):
// state = [n, mean0 (p_0), C^(0..k_max) packed], float64, host memory.
// ---------------------------------------------------------------------------
static int64_t state_len(const std::vector<int> &p) {
    int64_t len = 1 + p[0];
    for (int v : p) len += (int64_t)v * v;
    return len;
}

extern "C" int ffb_cov_export(ffb_plan_t p, double *h_state, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !h_state) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    CK(ffb_launch_cov_final(p, s));
    h_state[0] = (double)p->n_acc;
    CK(ffb_check_cuda(cudaMemcpyAsync(h_state + 1, p->d_mean, sizeof(double) * p->p[0], cudaMemcpyDeviceToHost, s)));
    CK(ffb_check_cuda(cudaMemcpyAsync(h_state + 1 + p->p[0], p->d_Cfin, sizeof(double) * p->cov_total,
                                      cudaMemcpyDeviceToHost, s)));
    return read_status(p, s);
}

// Pooled statistics of nstates disjoint image sets (Chan et al.'s pairwise
// update generalised): n = sum n_r, m = sum n_r m_r / n,
// C^(0) = sum n_r (C0_r + (m_r - m)(m_r - m)^T) / n, C^(k>0) = sum n_r C^(k)_r / n.
extern "C" int ffb_cov_merge(int k_max, const int *h_p, int nstates, const double *h_states, double *h_out) {
    if (k_max < 0 || !h_p || nstates < 1 || !h_states || !h_out) return FFB_ERR_ARG;
    std::vector<int> p(h_p, h_p + k_max + 1);
    for (int v : p)
        if (v <= 0) return FFB_ERR_ARG;
    const int64_t len = state_len(p);
    const int p0 = p[0];
    double n = 0.0;
    for (int r = 0; r < nstates; ++r) {
        const double nr = h_states[(size_t)r * len];
        if (!(nr > 0.0)) return FFB_ERR_ARG;
        n += nr;
    }
    std::vector<double> out((size_t)len, 0.0);
    out[0] = n;
    for (int r = 0; r < nstates; ++r) {
        const double *st = h_states + (size_t)r * len;
        for (int q = 0; q < p0; ++q) out[1 + q] += st[0] * st[1 + q] / n;
    }
    for (int r = 0; r < nstates; ++r) {
        const double *st = h_states + (size_t)r * len;
        const double w = st[0] / n;
        const double *mr = st + 1;
        // k = 0 block with the between-set term
        for (int a = 0; a < p0; ++a)
            for (int b = 0; b < p0; ++b) {
                const double da = mr[a] - out[1 + a], db = mr[b] - out[1 + b];
                out[1 + p0 + (size_t)a * p0 + b] += w * (st[1 + p0 + (size_t)a * p0 + b] + da * db);
            }
        for (int64_t e = 1 + p0 + (int64_t)p0 * p0; e < len; ++e) out[(size_t)e] += w * st[e];
    }
    std::copy(out.begin(), out.end(), h_out);
    return FFB_OK;
}

// Loads pooled statistics into the plan's accumulator (shift = rounded mean),
// after which ffb_cov_get / ffb_eig see the pooled covariance.
extern "C" int ffb_cov_import(ffb_plan_t p, const double *h_state, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || !h_state || !(h_state[0] >= 1.0)) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int p0 = p->p[0];
    const double n = h_state[0];
    std::vector<float> shift(p0);
    std::vector<double> sum0(p0), acc(p->cov_total);
    for (int q = 0; q < p0; ++q) {
        shift[q] = (float)h_state[1 + q];
        sum0[q] = n * (h_state[1 + q] - (double)shift[q]);
    }
    const double *C = h_state + 1 + p0;
    for (int a = 0; a < p0; ++a)
        for (int b = 0; b < p0; ++b)
            acc[(size_t)a * p0 + b] = n * (C[(size_t)a * p0 + b] + (sum0[a] / n) * (sum0[b] / n));
    for (int e = p0 * p0; e < p->cov_total; ++e) acc[e] = n * C[e];
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_shift, shift.data(), sizeof(float) * p0, cudaMemcpyHostToDevice, s)));
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_sum0, sum0.data(), sizeof(double) * p0, cudaMemcpyHostToDevice, s)));
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_acc, acc.data(), sizeof(double) * p->cov_total, cudaMemcpyHostToDevice, s)));
    CK(ffb_check_cuda(cudaStreamSynchronize(s)));
    p->n_acc = (int64_t)(n + 0.5);
    p->shift_set = 1;
    return FFB_OK;
}
