// ffb_api.cu -- C ABI entry points of the hot path (see include/ffb.h).
#include <algorithm>

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
    if (!p) return FFB_ERR_ARG;
    return read_status(p, (cudaStream_t)stream);
}

extern "C" int ffb_profile(ffb_plan_t p, int enable) {
    if (!p) return FFB_ERR_ARG;
    p->prof_on = enable ? 1 : 0;
    p->prof_used = 0;
    return FFB_OK;
}

extern "C" int ffb_profile_read(ffb_plan_t p, double *h_ms, int64_t *h_calls) {
    if (!p || !h_ms || !h_calls) return FFB_ERR_ARG;
    for (int c = 0; c < FFB_NKC; ++c) {
        h_ms[c] = 0.0;
        h_calls[c] = 0;
    }
    for (size_t i = 0; i < p->prof_used; ++i) {
        const ProfEv &e = p->prof[i];
        if (cudaEventSynchronize(e.b) != cudaSuccess) return FFB_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) != cudaSuccess) return FFB_ERR_CUDA;
        h_ms[e.cls] += ms;
        h_calls[e.cls] += 1;
    }
    p->prof_used = 0;
    return FFB_OK;
}

extern "C" int ffb_polar(ffb_plan_t p, const float *d_images, int64_t n, float *d_F, void *stream) {
    if (!p || n < 0 || (n > 0 && (!d_images || !d_F))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(ffb_ensure_scratch(p));
    const size_t per = (size_t)p->n_xi * (p->n_theta / 2) * 2;
    for (int64_t i0 = 0; i0 < n; i0 += p->chunk) {
        int m = (int)std::min<int64_t>(p->chunk, n - i0);
        CK(ffb_launch_grid(p, d_images, i0, m, s));
        CK(ffb_launch_polar(p, m, d_F + (size_t)i0 * per, s));
    }
    return FFB_OK;
}

extern "C" int ffb_expand(ffb_plan_t p, const float *d_images, int64_t n, float *d_coef, void *stream) {
    if (!p || n < 0 || (n > 0 && (!d_images || !d_coef))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(ffb_ensure_scratch(p));
    for (int64_t i0 = 0; i0 < n; i0 += p->chunk) {
        int m = (int)std::min<int64_t>(p->chunk, n - i0);
        CK(ffb_launch_grid(p, d_images, i0, m, s));
        CK(ffb_launch_interp_ring(p, m, s));
        CK(ffb_launch_bessel(p, m, d_coef + (size_t)i0 * p->P * 2, s));
    }
    return FFB_OK;
}

extern "C" int ffb_covariance(ffb_plan_t p, const float *d_coef, int64_t n, int reset, void *stream) {
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

extern "C" int ffb_eig(ffb_plan_t p, double *d_evals, double *d_evecs, void *stream) {
    if (!p) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    CK(ffb_launch_cov_final(p, s));
    CK(ffb_launch_eig(p, s));
    if (d_evals)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evals, p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, s)));
    if (d_evecs)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evecs, p->d_evecs, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    return read_status(p, s);
}

extern "C" int ffb_eig_blocks(ffb_plan_t p, const double *d_C, double *d_evals, double *d_evecs, void *stream) {
    if (!p || !d_C) return FFB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(ffb_check_cuda(cudaMemcpyAsync(p->d_Cfin, d_C, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    CK(ffb_launch_eig(p, s));
    if (d_evals)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evals, p->d_evals, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, s)));
    if (d_evecs)
        CK(ffb_check_cuda(cudaMemcpyAsync(d_evecs, p->d_evecs, sizeof(double) * p->cov_total, cudaMemcpyDeviceToDevice, s)));
    return read_status(p, s);
}

extern "C" int ffb_expand_adjoint(ffb_plan_t p, const float *d_coef, int64_t n, float *d_images, void *stream) {
    if (!p || n < 0 || (n > 0 && (!d_coef || !d_images))) return FFB_ERR_ARG;
    if (n == 0) return FFB_OK;
    return ffb_launch_adjoint(p, d_coef, n, d_images, (cudaStream_t)stream);
}

extern "C" int ffb_denoise(ffb_plan_t p, const float *d_images, int64_t n, int mode, int K, double sigma2,
                           float *d_out, void *stream) {
    (void)p; (void)d_images; (void)n; (void)mode; (void)K; (void)sigma2; (void)d_out; (void)stream;
    return FFB_ERR_UNSUPPORTED;
}

int ffb_launch_adjoint(ffb_plan_t p, const float *d_coef, int64_t n, float *d_images, cudaStream_t s) {
    (void)p; (void)d_coef; (void)n; (void)d_images; (void)s;
    return FFB_ERR_UNSUPPORTED;
}
