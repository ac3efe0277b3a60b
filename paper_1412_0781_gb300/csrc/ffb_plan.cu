// ffb_plan.cu -- Alg. 1 steps 1-2 (precomputation) on the GPU in float64:
// Bessel zeros R_{k,q}, the sampling criterion (Eq. criterion1), the
// Gauss-Legendre rule on [0, c], the radial table of Eq. a, and the NUFFT
// tables (kernel deconvolution, FFT twiddles, polar node coordinates).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ffb_internal.cuh"

// ---------------------------------------------------------------------------
// float64 special functions (device)
// ---------------------------------------------------------------------------

// Bessel zeros: one block per order k scans [lo, X + 2 step] on a grid of
// spacing `step` (< the 2.4 minimum gap between positive zeros), brackets
// sign changes, ranks the brackets and refines each by bisection.  Writes
// zeros[k * qcap + q] ascending and count[k] = number of zeros <= X.
__global__ void k_bessel_zeros(double X, double step, int qcap, double *zeros, int *count,
                               int *status) {
    extern __shared__ double sh[];
    const int k = blockIdx.x;
    const double lo = (k == 0) ? 1e-3 : (double)k;
    __shared__ int nbr;
    __shared__ int brk[1024];
    const int ngrid = (int)ceil((X + 2.0 * step - lo) / step) + 1;
    if (threadIdx.x == 0) nbr = 0;
    if (ngrid <= 1 || lo >= X) {
        if (threadIdx.x == 0) count[k] = 0;
        return;
    }
    __syncthreads();
    double *v = sh;  // ngrid values
    for (int i = threadIdx.x; i < ngrid; i += blockDim.x) v[i] = bessel_j_miller(k, lo + step * i);
    __syncthreads();
    for (int i = threadIdx.x; i + 1 < ngrid; i += blockDim.x) {
        if ((v[i] < 0.0) != (v[i + 1] < 0.0) && v[i] != 0.0) {
            int slot = atomicAdd(&nbr, 1);
            if (slot < 1024) brk[slot] = i;
        }
    }
    __syncthreads();
    const int nb = min(nbr, 1024);
    if (nbr > 1024 || nb > qcap) {
        if (threadIdx.x == 0) ffb_flag(status, FFB_ERR_UNSUPPORTED);
        return;
    }
    if (threadIdx.x == 0) count[k] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int i = brk[b];
        int rank = 0;
        for (int c = 0; c < nb; ++c) rank += (brk[c] < i);
        double a = lo + step * i, bb = a + step;
        double fa = v[i];
        for (int it = 0; it < 60; ++it) {
            double m = 0.5 * (a + bb);
            double fm = bessel_j_miller(k, m);
            if ((fm < 0.0) == (fa < 0.0)) {
                a = m;
                fa = fm;
            } else {
                bb = m;
            }
        }
        double z = 0.5 * (a + bb);
        zeros[(size_t)k * qcap + rank] = z;
        if (z <= X) atomicAdd(&count[k], 1);
    }
}

// n-point Gauss-Legendre rule on [a, b]: Newton iteration on P_n (three-term
// recurrence) from x ~ cos(pi (i + 3/4) / (n + 1/2)); weights
// 2 / ((1 - x^2) P_n'(x)^2).  Node index ascending in [a, b].
__global__ void k_gauss_legendre(int n, double a, double b, double *x_out, double *w_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double pi = 3.14159265358979323846;
    double x = cos(pi * (i + 0.75) / (n + 0.5));  // descending in i
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int m = 1; m < n; ++m) {
            double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (p0 - x * p1) / (1.0 - x * x);
        double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16 && it > 2) break;
    }
    {
        double p0 = 1.0, p1 = x;
        for (int m = 1; m < n; ++m) {
            double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (p0 - x * p1) / (1.0 - x * x);
    }
    double w = 2.0 / ((1.0 - x * x) * dp * dp);
    int j = n - 1 - i;  // ascending order
    double half = 0.5 * (b - a);
    x_out[j] = a + half * (x + 1.0);
    w_out[j] = half * w;
}

// B^(k)_{q,j} = N_{k,q} J_k(R_{k,q} xi_j / c) xi_j w_j, N_{k,q} =
// 1 / (c sqrt(pi) |J_{k+1}(R_{k,q})|)   (Eq. FB and Eq. a).
__global__ void k_bessel_table(int P, int n_xi, double c, const double *zeros, const int *kof,
                               const double *xi, const double *wq, double *B64, float *Bf) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * n_xi) return;
    int idx = (int)(t / n_xi), j = (int)(t % n_xi);
    int k = kof[idx];
    double r = zeros[idx];
    const double sqrt_pi = 1.77245385090551602730;
    double nrm = 1.0 / (c * sqrt_pi * fabs(bessel_j_miller(k + 1, r)));
    double val = nrm * bessel_j_miller(k, r * xi[j] / c) * xi[j] * wq[j];
    B64[t] = val;
    Bf[t] = (float)val;
}

// Deconvolution of the interpolation kernel: corr[a] = 1 / Psi((a - off)/N),
// Psi(nu) = 2 int_0^{w/2} psi(x) cos(2 pi x nu) dx by Gauss-Legendre.
__global__ void k_es_correction(int L, int off, int N, int w, double beta, int ng,
                                const double *xg, const double *wg, float *corr) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= L) return;
    const double pi = 3.14159265358979323846;
    double nu = (double)(a - off) / N;
    double s = 0.0;
    for (int g = 0; g < ng; ++g) {
        double t = 2.0 * xg[g] / w;
        double psi = exp(beta * (sqrt(fmax(1.0 - t * t, 0.0)) - 1.0));
        s += wg[g] * psi * cos(2.0 * pi * xg[g] * nu);
    }
    corr[a] = (float)(1.0 / (2.0 * s));
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int ffb_check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return FFB_OK;
    if (e == cudaErrorMemoryAllocation) return FFB_ERR_OOM;
    return FFB_ERR_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        int _s = ffb_check_cuda(call);            \
        if (_s != FFB_OK) {                       \
            cudaGetLastError();                   \
            return _s;                            \
        }                                         \
    } while (0)

static bool factor_235(int n, FftPlanDev *fp) {
    fp->n = n;
    fp->nst = 0;
    int m = n;
    while (m % 4 == 0 && fp->nst < FFB_MAX_RADIX_STAGES) { fp->rad[fp->nst++] = 4; m /= 4; }
    while (m % 2 == 0 && fp->nst < FFB_MAX_RADIX_STAGES) { fp->rad[fp->nst++] = 2; m /= 2; }
    while (m % 3 == 0 && fp->nst < FFB_MAX_RADIX_STAGES) { fp->rad[fp->nst++] = 3; m /= 3; }
    while (m % 5 == 0 && fp->nst < FFB_MAX_RADIX_STAGES) { fp->rad[fp->nst++] = 5; m /= 5; }
    return m == 1;
}

template <class T>
static cudaError_t dalloc(T **p, size_t count) {
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// a temporary device buffer of plan construction, freed on every return path
struct ScopedDev {
    void *ptr = nullptr;
    ScopedDev() = default;
    ScopedDev(const ScopedDev &) = delete;
    ScopedDev &operator=(const ScopedDev &) = delete;
    ~ScopedDev() {
        if (ptr) cudaFree(ptr);
    }
};

static void free_plan(ffb_plan_t p) {
    ffb_tc_release(p);
    void *ptrs[] = {p->d_zeros, p->d_xi, p->d_wq, p->d_B64, p->d_Bf, p->d_p, p->d_off,
                    p->d_cov_off, p->d_corr, p->d_twN, p->d_twT, p->d_rad, p->d_ang,
                    p->d_cov_work, p->d_cov_sb, p->d_H, p->d_G, p->d_Fhat, p->d_acc, p->d_sum0,
                    p->d_shift, p->d_Cfin, p->d_mean, p->d_evals, p->d_evecs, p->d_status,
                    p->d_coef_den, p->d_gain, p->d_M, p->d_eig_work, p->d_Fpol, p->d_nodes, p->d_node_blk, p->d_twA, p->d_twG,
                    p->d_tunits, p->d_tblk, p->d_tnodes, p->d_hostimg, p->d_hostcoef};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < FFB_HOST_SLOTS; ++i) {
        if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
        if (p->ev_free[i]) cudaEventDestroy(p->ev_free[i]);
    }
    if (p->h2d) cudaStreamDestroy(p->h2d);
    for (ProfEv &e : p->prof) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete p;
}

static void twiddles(int n, std::vector<float2> &tw) {
    tw.resize(n);
    for (int e = 0; e < n; ++e) {
        double ang = -2.0 * M_PI * (double)e / (double)n;
        tw[e] = make_float2((float)cos(ang), (float)sin(ang));
    }
}

static int build_plan(ffb_plan_t p, cudaStream_t s) {
    const double X = 2.0 * M_PI * p->c * p->R;  // right-hand side of Eq. criterion1
    // ---- Bessel zeros and the sampling criterion -------------------------
    const int kcand = (int)floor(X) + 2;
    const int qcap = (int)floor(X / M_PI) + 4;
    const double step = 0.25;
    ScopedDev tz, tc;
    CK(cudaMalloc(&tz.ptr, sizeof(double) * (size_t)kcand * qcap));
    CK(cudaMalloc(&tc.ptr, sizeof(int) * kcand));
    double *d_z = (double *)tz.ptr;
    int *d_cnt = (int *)tc.ptr;
    int ngrid_max = (int)ceil((X + 2.0 * step) / step) + 2;
    size_t shm = sizeof(double) * (size_t)ngrid_max;
    if (shm > 48 * 1024) CK(cudaFuncSetAttribute(k_bessel_zeros, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_bessel_zeros<<<kcand, 128, shm, s>>>(X, step, qcap, d_z, d_cnt, p->d_status);
    p->launches++;
    CK(cudaGetLastError());
    std::vector<double> hz((size_t)kcand * qcap);
    std::vector<int> hc(kcand);
    CK(cudaMemcpyAsync(hz.data(), d_z, hz.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hc.data(), d_cnt, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    int hstatus = 0;
    CK(cudaMemcpyAsync(&hstatus, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hstatus != 0) return hstatus;
    std::vector<double> zsel;
    std::vector<int> kof;
    p->p.clear();
    for (int k = 0; k < kcand; ++k) {
        int pk = hc[k] - 1;  // literal criterion: R_{k,q+1} <= 2 pi c R
        if (pk <= 0) break;
        p->p.push_back(pk);
        for (int q = 0; q < pk; ++q) {
            zsel.push_back(hz[(size_t)k * qcap + q]);
            kof.push_back(k);
        }
    }
    if (p->p.empty()) return FFB_ERR_ARG;
    p->k_max = (int)p->p.size() - 1;
    p->P = (int)zsel.size();
    p->offset.resize(p->k_max + 1);
    p->cov_off.resize(p->k_max + 2);
    p->pmax = 0;
    int o = 0, co = 0;
    for (int k = 0; k <= p->k_max; ++k) {
        p->offset[k] = o;
        p->cov_off[k] = co;
        o += p->p[k];
        co += p->p[k] * p->p[k];
        if (p->p[k] > p->pmax) p->pmax = p->p[k];
    }
    p->cov_off[p->k_max + 1] = co;
    p->cov_total = co;

    // ---- device copies of the selection ---------------------------------
    ScopedDev tk;
    CK(dalloc(&p->d_zeros, p->P));
    CK(cudaMalloc(&tk.ptr, sizeof(int) * (size_t)std::max(p->P, 1)));
    int *d_kof = (int *)tk.ptr;
    CK(dalloc(&p->d_p, p->k_max + 1));
    CK(dalloc(&p->d_off, p->k_max + 1));
    CK(dalloc(&p->d_cov_off, p->k_max + 2));
    CK(cudaMemcpyAsync(p->d_zeros, zsel.data(), sizeof(double) * p->P, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_kof, kof.data(), sizeof(int) * p->P, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_p, p->p.data(), sizeof(int) * (p->k_max + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_off, p->offset.data(), sizeof(int) * (p->k_max + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_cov_off, p->cov_off.data(), sizeof(int) * (p->k_max + 2), cudaMemcpyHostToDevice, s));

    // ---- Gauss-Legendre rule on [0, c] and the radial table -----------------
    CK(dalloc(&p->d_xi, p->n_xi));
    CK(dalloc(&p->d_wq, p->n_xi));
    k_gauss_legendre<<<(p->n_xi + 127) / 128, 128, 0, s>>>(p->n_xi, 0.0, p->c, p->d_xi, p->d_wq);
    p->launches++;
    CK(cudaGetLastError());
    CK(dalloc(&p->d_B64, (size_t)p->P * p->n_xi));
    CK(dalloc(&p->d_Bf, (size_t)p->P * p->n_xi));
    {
        int64_t tot = (int64_t)p->P * p->n_xi;
        k_bessel_table<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(p->P, p->n_xi, p->c, p->d_zeros, d_kof,
                                                                     p->d_xi, p->d_wq, p->d_B64, p->d_Bf);
        p->launches++;
        CK(cudaGetLastError());
    }

    // ---- NUFFT kernel deconvolution ------------------------------------
    {
        const int ng = 256;
        ScopedDev txg, twg;
        CK(cudaMalloc(&txg.ptr, sizeof(double) * ng));
        CK(cudaMalloc(&twg.ptr, sizeof(double) * ng));
        double *d_xg = (double *)txg.ptr, *d_wg = (double *)twg.ptr;
        k_gauss_legendre<<<(ng + 127) / 128, 128, 0, s>>>(ng, 0.0, 0.5 * p->w, d_xg, d_wg);
        p->launches++;
        CK(dalloc(&p->d_corr, p->L));
        k_es_correction<<<(p->L + 127) / 128, 128, 0, s>>>(p->L, p->off, p->N, p->w, p->beta, ng, d_xg,
                                                            d_wg, p->d_corr);
        p->launches++;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    }

    // ---- FFT twiddles, polar node coordinates --------------------------
    std::vector<float2> tw;
    twiddles(p->N, tw);
    CK(dalloc(&p->d_twN, p->N));
    CK(cudaMemcpyAsync(p->d_twN, tw.data(), sizeof(float2) * p->N, cudaMemcpyHostToDevice, s));
    std::vector<float2> twt;
    twiddles(p->n_theta, twt);
    CK(dalloc(&p->d_twT, p->n_theta));
    CK(cudaMemcpyAsync(p->d_twT, twt.data(), sizeof(float2) * p->n_theta, cudaMemcpyHostToDevice, s));
    std::vector<double> hxi(p->n_xi);
    CK(cudaMemcpyAsync(hxi.data(), p->d_xi, sizeof(double) * p->n_xi, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<float2> hrad(p->n_xi);
    for (int j = 0; j < p->n_xi; ++j) {
        double v = (double)p->N * hxi[j];
        float hi = (float)v;
        hrad[j] = make_float2(hi, (float)(v - (double)hi));
    }
    const int nh = p->n_theta / 2;
    std::vector<float4> hang(nh);
    for (int l = 0; l < nh; ++l) {
        double th = 2.0 * M_PI * (double)l / (double)p->n_theta;
        double cv = cos(th), sv = sin(th);
        float ch = (float)cv, sh2 = (float)sv;
        hang[l] = make_float4(ch, (float)(cv - (double)ch), sh2, (float)(sv - (double)sh2));
    }
    CK(dalloc(&p->d_rad, p->n_xi));
    CK(dalloc(&p->d_ang, nh));
    CK(cudaMemcpyAsync(p->d_rad, hrad.data(), sizeof(float2) * p->n_xi, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_ang, hang.data(), sizeof(float4) * nh, cudaMemcpyHostToDevice, s));

    // ---- covariance work list: (k, q0, q0') tiles of 64 x 64 ------------
    std::vector<int4> work;
    for (int k = 0; k <= p->k_max; ++k)
        for (int q0 = 0; q0 < p->p[k]; q0 += 64)
            for (int q1 = q0; q1 < p->p[k]; q1 += 64) work.push_back(make_int4(k, q0, q1, 0));
    p->n_cov_work = (int)work.size();
    CK(dalloc(&p->d_cov_work, work.size()));
    CK(cudaMemcpyAsync(p->d_cov_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice, s));
    // tensor-core covariance super-blocks: runs of consecutive k with
    // sum p_k <= 128, as (first k, end k, first coefficient index, rows)
    std::vector<int4> sbs;
    for (int k = 0; k <= p->k_max;) {
        int rows = 0, k1 = k;
        while (k1 <= p->k_max && (k1 == k || rows + p->p[k1] <= 128)) rows += p->p[k1++];
        sbs.push_back(make_int4(k, k1, p->offset[k], rows));
        k = k1;
    }
    p->n_cov_sb = (int)sbs.size();
    CK(dalloc(&p->d_cov_sb, sbs.size()));
    CK(cudaMemcpyAsync(p->d_cov_sb, sbs.data(), sizeof(int4) * sbs.size(), cudaMemcpyHostToDevice, s));

    // ---- covariance state and eig outputs ------------------------------
    CK(dalloc(&p->d_acc, p->cov_total));
    CK(dalloc(&p->d_sum0, p->p[0]));
    CK(dalloc(&p->d_shift, p->p[0]));
    CK(dalloc(&p->d_Cfin, p->cov_total));
    CK(dalloc(&p->d_mean, p->p[0]));
    CK(dalloc(&p->d_evals, p->P));
    CK(dalloc(&p->d_evecs, p->cov_total));
    CK(cudaMemsetAsync(p->d_acc, 0, sizeof(double) * p->cov_total, s));
    CK(cudaMemsetAsync(p->d_sum0, 0, sizeof(double) * p->p[0], s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(&hstatus, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    return hstatus;
}

// row spectra and half grid of a chunk (separate-kernel NUFFT and adjoint)
bool ffb_ring_buffers_fit(int n_theta, int rb) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return sizeof(float2) * 2 * (size_t)rb * n_theta <= (size_t)optin;
}

int ffb_ensure_scratch_grid(ffb_plan_t p) {
    if (!p->d_H) CK(dalloc(&p->d_H, (size_t)p->chunk * (p->N / 2 + 1) * p->L));
    if (!p->d_G) CK(dalloc(&p->d_G, (size_t)p->chunk * p->Mh * p->N));
    // the tiled interpolation writes polar samples before the ring DFTs
    if (p->ntblk > 0 && !p->d_Fpol) CK(dalloc(&p->d_Fpol, (size_t)p->chunk * p->n_xi * (p->n_theta / 2)));
    return FFB_OK;
}

// ring spectra of a chunk, plus the polar samples (fused path) or the grid
int ffb_ensure_scratch(ffb_plan_t p) {
    if (!p->d_Fhat) CK(dalloc(&p->d_Fhat, (size_t)(p->k_max + 1) * p->chunk * 2 * p->n_xi));
    if (p->fused) {
        if (!p->d_Fpol) CK(dalloc(&p->d_Fpol, (size_t)p->chunk * p->n_xi * (p->n_theta / 2)));
        return FFB_OK;
    }
    return ffb_ensure_scratch_grid(p);
}

extern "C" int ffb_plan(ffb_plan_t *out, int L, double c, double R, double eps, int precision,
                        void *stream) {
    if (!out) return FFB_ERR_ARG;
    *out = nullptr;
    if (L < 8 || L > 512 || !(c > 0.0 && c <= 0.5) || !(R > 0.0 && R <= 0.5 * L) ||
        !(eps >= 1e-7 && eps <= 1e-2) || precision < FFB_FP32 || precision > FFB_TF32X3)
        return FFB_ERR_ARG;
    ffb_plan_t p = new (std::nothrow) ffb_plan_s();
    if (!p) return FFB_ERR_OOM;
    p->L = L;
    p->off = L / 2;
    p->c = c;
    p->R = R;
    p->eps = eps;
    p->precision = precision;
    p->n_xi = (int)ceil(4.0 * c * R - 1e-9);
    p->n_theta = (int)ceil(16.0 * c * R - 1e-9);
    p->n_theta += (p->n_theta & 1);  // the half-ring storage needs an even count
    p->N = 2 * L;
    p->w = (int)ceil(log10(1.0 / eps)) + 2;
    if (p->w < 4) p->w = 4;
    if (p->w > 16) p->w = 16;
    p->beta = 2.30 * p->w;
    p->h = (p->w + 1) / 2;
    p->Mh = p->N / 2 + 1 + 2 * p->h;
    p->chunk = 256;
    p->nq0 = p->n_theta / 4 + 1;   // l <= n_theta/4  <=>  cos(theta_l) >= 0
    if (!factor_235(p->N, &p->fftN) || !factor_235(p->n_theta, &p->fftT) || p->n_xi < 2) {
        delete p;
        return FFB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int st = ffb_check_cuda(cudaGetDevice(&p->device));
    if (st == FFB_OK) st = ffb_check_cuda(cudaMalloc(&p->d_status, sizeof(int)));
    if (st == FFB_OK) st = ffb_check_cuda(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    if (st == FFB_OK) st = build_plan(p, s);
    if (st == FFB_OK && p->precision != FFB_FP32 && !ffb_tc_supported(p)) st = FFB_ERR_UNSUPPORTED;
    if (st == FFB_OK && ffb_fused_supported(p)) {
        p->fused = ffb_fused_mode(p);
        p->chunk = 152;   // 2 x 152 CTAs of one per SM: two full waves on 152 SMs
        st = ffb_fused_prepare(p, s);
        if (st == FFB_OK) st = ffb_ring_prepare(p, s);
        p->ring_direct = 1;
    }
    if (st == FFB_OK && !p->fused) st = ffb_tile_prepare(p, s);
    // tiled plans whose ring length the register ring FFT takes
    const int nt = p->n_theta;
    if (st == FFB_OK && p->ntblk > 0 && (nt == 64 || nt == 128 || nt == 256 || nt == 512 || nt == 1024) &&
        p->k_max < nt / 2) {
        st = ffb_ring_prepare(p, s);
        p->ring_direct = (st == FFB_OK);
    }
    if (st != FFB_OK) {
        cudaStreamSynchronize(s);
        free_plan(p);
        return st;
    }
    *out = p;
    return FFB_OK;
}

extern "C" int ffb_plan_destroy(ffb_plan_t plan) {
    if (!plan) return FFB_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return FFB_OK;
}

extern "C" int ffb_plan_info(ffb_plan_t p, int *info) {
    if (!p || !info) return FFB_ERR_ARG;
    info[0] = p->L;
    info[1] = p->k_max;
    info[2] = p->P;
    info[3] = p->n_xi;
    info[4] = p->n_theta;
    info[5] = p->N;
    info[6] = p->w;
    info[7] = p->precision;
    info[8] = p->pmax;
    info[9] = p->chunk;
    info[10] = p->fused;
    return FFB_OK;
}

extern "C" int ffb_plan_sizes(ffb_plan_t p, int *h_p, int *h_offset) {
    if (!p) return FFB_ERR_ARG;
    for (int k = 0; k <= p->k_max; ++k) {
        if (h_p) h_p[k] = p->p[k];
        if (h_offset) h_offset[k] = p->offset[k];
    }
    return FFB_OK;
}

extern "C" int ffb_plan_tables(ffb_plan_t p, double *h_zeros, double *h_xi, double *h_w, double *h_B) {
    if (!p) return FFB_ERR_ARG;
    if (h_zeros) CK(cudaMemcpy(h_zeros, p->d_zeros, sizeof(double) * p->P, cudaMemcpyDeviceToHost));
    if (h_xi) CK(cudaMemcpy(h_xi, p->d_xi, sizeof(double) * p->n_xi, cudaMemcpyDeviceToHost));
    if (h_w) CK(cudaMemcpy(h_w, p->d_wq, sizeof(double) * p->n_xi, cudaMemcpyDeviceToHost));
    if (h_B) CK(cudaMemcpy(h_B, p->d_B64, sizeof(double) * (size_t)p->P * p->n_xi, cudaMemcpyDeviceToHost));
    return FFB_OK;
}

extern "C" int ffb_set_precision(ffb_plan_t p, int precision) {
    if (!p || precision < FFB_FP32 || precision > FFB_TF32X3) return FFB_ERR_ARG;
    const int old = p->precision;
    p->precision = precision;
    if (precision != FFB_FP32 && !ffb_tc_supported(p)) {
        p->precision = old;
        return FFB_ERR_UNSUPPORTED;
    }
    return FFB_OK;
}

int ffb_plan_here(ffb_plan_t p) {
    if (!p) return FFB_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FFB_ERR_CUDA;
    }
    return dev == p->device ? FFB_OK : FFB_ERR_ARG;
}

extern "C" int ffb_set_wait_budget(ffb_plan_t p, long long cycles) {
    if (!p) return FFB_ERR_ARG;
    p->wait_budget = (cycles < 0) ? FFB_WAIT_BUDGET : cycles;
    return FFB_OK;
}

extern "C" int64_t ffb_launch_count(ffb_plan_t p) { return p ? p->launches : 0; }

extern "C" const char *ffb_strerror(int status) {
    switch (status) {
        case FFB_OK: return "ok";
        case FFB_ERR_ARG: return "invalid argument";
        case FFB_ERR_CUDA: return "CUDA runtime error";
        case FFB_ERR_OOM: return "device out of memory";
        case FFB_ERR_NONFINITE: return "non-finite value in input";
        case FFB_ERR_NOT_CONVERGED: return "Jacobi eigensolver did not converge";
        case FFB_ERR_TIMEOUT: return "device-side wait timed out";
        case FFB_ERR_STATE: return "call out of order";
        case FFB_ERR_UNSUPPORTED: return "unsupported size or precision";
        default: return "unknown status";
    }
}
