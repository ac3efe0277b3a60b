// ffb_nufft.cu -- steps a1-a4 of the hot path (Alg. 1 steps 3-4):
// the polar Fourier transform of Eq. nufft by a type-2 NUFFT (precorrect,
// oversampled 2D FFT, kernel interpolation) and the angular DFT of Eq. 1DFFT
// on every ring.
//
// Fine grid.  With N = 2L and the exponential-of-semicircle kernel psi of
// width w (Fourier transform Psi), Poisson summation gives
//   e^{-2 pi i xi i} ~ (1/Psi(i/N)) sum_m psi(N xi - m) e^{-2 pi i m i / N},
// so F(xi) = sum_i I(i) e^{-2 pi i xi.i} ~ sum_{m1,m2} psi(N xi1 - m1)
// psi(N xi2 - m2) G[m1][m2] with G the N x N DFT of I(i)/(Psi(i1/N)Psi(i2/N))
// placed at (i1 mod N, i2 mod N).  Images are real, so G[-m] = conj G[m] and
// only m2 in [-h, N/2 + h] is kept (h = ceil(w/2) halo rows filled by that
// symmetry); the polar nodes used have theta in [0, pi), i.e. xi2 >= 0, and
// the other half ring is the complex conjugate.
//
// Layouts (per image of the chunk):
//   H [N/2+1][L]  row transform: H[m2][a1] = sum_{i2} I'(a1, i2) e^{-2 pi i m2 i2/N}
//   G [Mh][N]     G[m2 + h][m1], Mh = N/2 + 1 + 2h
//   Fhat [k][img][c][j]  (2 pi / n_theta) * ring DFT, c = re/im, k <= k_max
#include "ffb_internal.cuh"

#define ROW_WARPS 8
#define COL_WARPS 8
#define RING_RB 8
#define RING_NT 256

// ---------------------------------------------------------------------------
// a1 + a2 (rows): precorrection, placement at i2 mod N, two real rows packed
// into one complex FFT of length N, unpacked into the half spectrum.
// grid (ceil(L / 2 ROW_WARPS), nimg), block 32 ROW_WARPS
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * ROW_WARPS)
k_rows(const float *__restrict__ images, int L, int off, int N, const float *__restrict__ corr,
       const float2 *__restrict__ tw, FftPlanDev fp, float2 *__restrict__ H, int *status) {
    extern __shared__ float2 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int img = blockIdx.y;
    const int a1b = blockIdx.x * 2 * ROW_WARPS;
    const int a1 = a1b + 2 * warp;
    const int Nh = N / 2 + 1;
    float2 *bufA = sm + warp * 2 * N;
    float2 *bufB = bufA + N;
    float2 *stage = sm + ROW_WARPS * 2 * N;  // [Nh][2 ROW_WARPS]
    const float *im = images + (size_t)img * L * L;
    for (int q = lane; q < N; q += 32) bufA[q] = make_float2(0.f, 0.f);
    __syncwarp();
    bool bad = false;
    if (a1 < L) {
        const bool two = (a1 + 1) < L;
        const float c1 = corr[a1];
        const float c2 = two ? corr[a1 + 1] : 0.f;
        for (int a2 = lane; a2 < L; a2 += 32) {
            float x = __ldg(&im[(size_t)a1 * L + a2]);
            float y = two ? __ldg(&im[(size_t)(a1 + 1) * L + a2]) : 0.f;
            bad |= !(isfinite(x) && isfinite(y));
            int pos = a2 - off;
            if (pos < 0) pos += N;
            float ca = corr[a2];
            bufA[pos] = make_float2(x * c1 * ca, y * c2 * ca);
        }
    }
    if (bad) ffb_flag(status, FFB_ERR_NONFINITE);
    __syncwarp();
    float2 *X = smem_fft<false>(bufA, bufB, fp, tw, lane, 32, WarpSync());
    for (int m = lane; m < Nh; m += 32) {
        float2 Z = X[m];
        float2 Zc = cconj(X[m == 0 ? 0 : N - m]);
        float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
        float2 D = csub(Z, Zc);
        float2 B = make_float2(0.5f * D.y, -0.5f * D.x);  // (Z - Zc) / 2i
        stage[m * 2 * ROW_WARPS + 2 * warp] = A;
        stage[m * 2 * ROW_WARPS + 2 * warp + 1] = B;
    }
    __syncthreads();
    float2 *Hi = H + (size_t)img * Nh * L;
    for (int idx = threadIdx.x; idx < Nh * 2 * ROW_WARPS; idx += blockDim.x) {
        int m = idx / (2 * ROW_WARPS), r = idx % (2 * ROW_WARPS);
        int a = a1b + r;
        if (a < L) Hi[(size_t)m * L + a] = stage[idx];
    }
}

// ---------------------------------------------------------------------------
// a2 (columns): for every m2 in [0, N/2] the length-N transform over i1,
// written to G[m2 + h][.]; rows h - m2 (m2 = 1..h) and h + N - m2
// (m2 = N/2 - h .. N/2 - 1) receive conj G[-m1][m2] (Hermitian halo).
// grid (ceil((N/2+1) / COL_WARPS), nimg), block 32 COL_WARPS
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * COL_WARPS)
k_cols(const float2 *__restrict__ H, int L, int off, int N, int h, int Mh,
       const float2 *__restrict__ tw, FftPlanDev fp, float2 *__restrict__ G) {
    extern __shared__ float2 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int img = blockIdx.y;
    const int Nh = N / 2 + 1;
    const int m2 = blockIdx.x * COL_WARPS + warp;
    if (m2 >= Nh) return;  // no block-wide barrier below
    float2 *bufA = sm + warp * 2 * N;
    float2 *bufB = bufA + N;
    for (int q = lane; q < N; q += 32) bufA[q] = make_float2(0.f, 0.f);
    __syncwarp();
    const float2 *Hc = H + ((size_t)img * Nh + m2) * L;
    for (int a1 = lane; a1 < L; a1 += 32) {
        int pos = a1 - off;
        if (pos < 0) pos += N;
        bufA[pos] = Hc[a1];
    }
    __syncwarp();
    float2 *X = smem_fft<false>(bufA, bufB, fp, tw, lane, 32, WarpSync());
    float2 *Gi = G + (size_t)img * Mh * N;
    float2 *row = Gi + (size_t)(m2 + h) * N;
    for (int m1 = lane; m1 < N; m1 += 32) row[m1] = X[m1];
    if (m2 >= 1 && m2 <= h) {
        float2 *er = Gi + (size_t)(h - m2) * N;
        for (int m1 = lane; m1 < N; m1 += 32) er[m1] = cconj(X[m1 == 0 ? 0 : N - m1]);
    }
    if (m2 >= 1 && m2 >= N / 2 - h && m2 <= N / 2 - 1) {
        float2 *er = Gi + (size_t)(h + N - m2) * N;
        for (int m1 = lane; m1 < N; m1 += 32) er[m1] = cconj(X[m1 == 0 ? 0 : N - m1]);
    }
}

// ---------------------------------------------------------------------------
// a3 + a4: interpolation at the half-ring nodes of RB rings and the
// length-n_theta ring FFT (Eq. 1DFFT) with F(theta + pi) = conj F(theta).
// POLAR = true writes the interpolated half rings (ffb_polar) instead.
// grid (ceil(n_xi / RB), nimg), block RING_NT
//
// Node coordinates t = N xi_j cos(theta_l) are formed in double-float
// (hi + lo parts) so that the stencil offset f = t - m0 keeps ~1e-7 absolute
// accuracy even where t ~ N/2: rounding xi to float32 alone would move the
// node by ~3e-8 and the phase of F by 2 pi * 3e-8 * |i|.
// ---------------------------------------------------------------------------
// FROM_POLAR: the half rings come from the polar buffer Fpolar (written by
// the tiled interpolation of ffb_tile.cu) instead of being interpolated here.
template <bool POLAR, int RB, bool FROM_POLAR = false>
__global__ void __launch_bounds__(RING_NT)
k_interp_ring(const float2 *__restrict__ G, int N, int h, int Mh, int w, float beta,
              const float2 *__restrict__ rad, const float4 *__restrict__ ang, int n_xi, int n_theta,
              const float2 *__restrict__ twT, FftPlanDev fpT, int kmax, int chunk,
              float *__restrict__ Fhat, float2 *__restrict__ Fpolar, int *status) {
    extern __shared__ float2 sm[];
    float2 *ringA = sm;                         // [RB][n_theta]
    float2 *ringB = sm + RB * n_theta;     // [RB][n_theta]
    const int img = blockIdx.y;
    const int j0 = blockIdx.x * RB;
    const int nh = n_theta / 2;
    const float2 *Gi = G + (size_t)img * Mh * N;
    const float halfw = 0.5f * (float)w;
    const float two_over_w = 2.0f / (float)w;
    for (int t = threadIdx.x; t < RB * nh; t += RING_NT) {
        const int jj = t / nh, l = t - jj * nh;
        const int j = j0 + jj;
        float2 val = make_float2(0.f, 0.f);
        if (FROM_POLAR) {
            if (j < n_xi) val = __ldg(&Fpolar[((size_t)img * n_xi + j) * nh + l]);
        } else if (j < n_xi) {
            const float2 r = __ldg(&rad[j]);
            const float4 a = __ldg(&ang[l]);
            float p1 = r.x * a.x;
            float e1 = fmaf(r.x, a.x, -p1) + fmaf(r.x, a.y, r.y * a.x);
            float p2 = r.x * a.z;
            float e2 = fmaf(r.x, a.z, -p2) + fmaf(r.x, a.w, r.y * a.z);
            float m1f = ceilf(p1 - halfw), m2f = ceilf(p2 - halfw);
            float f1 = (p1 - m1f) + e1, f2 = (p2 - m2f) + e2;
            int m1 = (int)m1f, m2 = (int)m2f;
            if (m2 + h < 0 || m2 + w - 1 + h >= Mh || m1 < -N || m1 > N) {
                ffb_flag(status, FFB_ERR_ARG);
            } else {
                float wx[16];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q < w) wx[q] = es_kernel(f1 - (float)q, two_over_w, beta);
                for (int b = 0; b < w; ++b) {
                    const float wy = es_kernel(f2 - (float)b, two_over_w, beta);
                    const float2 *row = Gi + (size_t)(m2 + b + h) * N;
                    float sx = 0.f, sy = 0.f;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if (q < w) {
                            int mm = m1 + q;
                            if (mm < 0) mm += N;
                            else if (mm >= N) mm -= N;
                            float2 g = __ldg(&row[mm]);
                            sx = fmaf(wx[q], g.x, sx);
                            sy = fmaf(wx[q], g.y, sy);
                        }
                    }
                    val.x = fmaf(wy, sx, val.x);
                    val.y = fmaf(wy, sy, val.y);
                }
            }
        }
        if (POLAR && !FROM_POLAR) {
            if (j < n_xi) Fpolar[((size_t)img * n_xi + j) * nh + l] = val;
        } else {
            ringA[jj * n_theta + l] = val;
            ringA[jj * n_theta + l + nh] = cconj(val);
        }
    }
    if (POLAR) return;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int jj = warp; jj < RB; jj += RING_NT / 32)
        smem_fft<false>(ringA + jj * n_theta, ringB + jj * n_theta, fpT, twT, lane, 32, WarpSync());
    __syncthreads();
    const float2 *res = (fpT.nst & 1) ? ringB : ringA;
    const float scale = 6.283185307179586f / (float)n_theta;
    const int tot = (kmax + 1) * 2 * RB;
    for (int t = threadIdx.x; t < tot; t += RING_NT) {
        const int jj = t % RB;
        const int cc = (t / RB) & 1;
        const int k = t / (2 * RB);
        const int j = j0 + jj;
        if (j < n_xi) {
            float2 v = res[jj * n_theta + k];
            Fhat[(((size_t)k * chunk + img) * 2 + cc) * n_xi + j] = scale * (cc ? v.y : v.x);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int ffb_launch_grid(ffb_plan_t p, const float *d_images, int64_t i0, int nimg, cudaStream_t s) {
    const int N = p->N, L = p->L, Nh = N / 2 + 1;
    size_t sm_rows = sizeof(float2) * ((size_t)ROW_WARPS * 2 * N + (size_t)Nh * 2 * ROW_WARPS);
    static int attr_rows = 0;
    if (sm_rows > 48 * 1024 && attr_rows < (int)sm_rows) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rows));
        if (e) return e;
        attr_rows = (int)sm_rows;
    }
    dim3 g1((L + 2 * ROW_WARPS - 1) / (2 * ROW_WARPS), nimg);
    {
    ProfScope ps(p, FFB_KC_ROWS, s);
    k_rows<<<g1, 32 * ROW_WARPS, sm_rows, s>>>(d_images + (size_t)i0 * L * L, L, p->off, N, p->d_corr,
                                                p->d_twN, p->fftN, p->d_H, p->d_status);
    p->launches++;
    }
    size_t sm_cols = sizeof(float2) * (size_t)COL_WARPS * 2 * N;
    static int attr_cols = 0;
    if (sm_cols > 48 * 1024 && attr_cols < (int)sm_cols) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cols));
        if (e) return e;
        attr_cols = (int)sm_cols;
    }
    dim3 g2((Nh + COL_WARPS - 1) / COL_WARPS, nimg);
    {
    ProfScope ps(p, FFB_KC_COLS, s);
    k_cols<<<g2, 32 * COL_WARPS, sm_cols, s>>>(p->d_H, L, p->off, N, p->h, p->Mh, p->d_twN, p->fftN, p->d_G);
    p->launches++;
    }
    return ffb_check_cuda(cudaGetLastError());
}

template <bool POLAR, int RB, bool FROM_POLAR = false>
static int launch_interp_rb(ffb_plan_t p, int nimg, float2 *d_F, cudaStream_t s) {
    size_t smem = (POLAR && !FROM_POLAR) ? 0 : sizeof(float2) * 2 * RB * (size_t)p->n_theta;
    static int attr = 0;
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_interp_ring<POLAR, RB, FROM_POLAR>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((p->n_xi + RB - 1) / RB, nimg);
    ProfScope ps(p, FROM_POLAR ? FFB_KC_RING_FFT : FFB_KC_INTERP, s);
    k_interp_ring<POLAR, RB, FROM_POLAR><<<g, RING_NT, smem, s>>>(p->d_G, p->N, p->h, p->Mh, p->w, (float)p->beta,
                                                                  p->d_rad, p->d_ang, p->n_xi, p->n_theta, p->d_twT,
                                                                  p->fftT, p->k_max, p->chunk, p->d_Fhat, d_F,
                                                                  p->d_status);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// RING_RB rings per CTA, or half as many where their two ring buffers would
// not fit in shared memory (n_theta > 1816 at 227 KB: L > 454 when R = L/2).
// Plans with a tile table interpolate with the tiled kernel (ffb_tile.cu)
// into the polar buffer, then take the ring DFTs from it.
template <bool POLAR>
static int launch_interp(ffb_plan_t p, int nimg, float2 *d_F, cudaStream_t s) {
    if (p->ntblk > 0) {
        if (POLAR) return ffb_launch_tile_polar(p, nimg, d_F, s);
        int e = ffb_launch_tile_polar(p, nimg, p->d_Fpol, s);
        if (e) return e;
        if (ffb_ring_buffers_fit(p->n_theta, RING_RB)) return launch_interp_rb<false, RING_RB, true>(p, nimg, p->d_Fpol, s);
        if (ffb_ring_buffers_fit(p->n_theta, RING_RB / 2))
            return launch_interp_rb<false, RING_RB / 2, true>(p, nimg, p->d_Fpol, s);
        return FFB_ERR_UNSUPPORTED;
    }
    if (POLAR || ffb_ring_buffers_fit(p->n_theta, RING_RB)) return launch_interp_rb<POLAR, RING_RB>(p, nimg, d_F, s);
    if (ffb_ring_buffers_fit(p->n_theta, RING_RB / 2)) return launch_interp_rb<POLAR, RING_RB / 2>(p, nimg, d_F, s);
    return FFB_ERR_UNSUPPORTED;
}

int ffb_launch_interp_ring(ffb_plan_t p, int nimg, cudaStream_t s) {
    return launch_interp<false>(p, nimg, nullptr, s);
}

int ffb_launch_polar(ffb_plan_t p, int nimg, float *d_F, cudaStream_t s) {
    return launch_interp<true>(p, nimg, (float2 *)d_F, s);
}

// ---------------------------------------------------------------------------
// ffb_polar_noalloc: the polar transform of ffb_polar without any device
// allocation, for callers that must not call cudaMalloc on the calling path:
// code running while a CUDA stream is being captured into a graph (where
// cudaMalloc is not allowed), real-time or serving loops whose latency budget
// cannot absorb an allocation, and host frameworks that own all device
// memory through their own pool and forbid third-party allocations.
//
// The scratch (row spectra and half grid of a group of images) lives in the
// file-scope array below, FFB_NOALLOC_SCRATCH_BYTES (16 MiB) per device,
// reserved for as long as the library stays loaded.  Host code cannot use the
// array's name as a device address; the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it, so that first call must come before any stream capture.  Every call
// shares the one array: calls that overlap on the GPU (different streams or
// host threads without ordering) race on it.  Each call writes every element
// it reads before reading it, so nothing has to start at zero.
// ---------------------------------------------------------------------------
#include <mutex>

#define FFB_NOALLOC_SCRATCH_BYTES (16u << 20)
#define FFB_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[FFB_NOALLOC_SCRATCH_BYTES];
static void *g_noalloc_addr[FFB_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

static int noalloc_scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FFB_ERR_CUDA;
    }
    if (dev < 0 || dev >= FFB_NOALLOC_MAX_DEVICES) return FFB_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) {
            cudaGetLastError();
            return FFB_ERR_CUDA;
        }
        g_noalloc_addr[dev] = addr;
    }
    *out = g_noalloc_addr[dev];
    return FFB_OK;
}

static int noalloc_smem(const void *fn, size_t bytes) {
    if (bytes <= 48 * 1024) return FFB_OK;
    return ffb_check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

extern "C" int ffb_polar_noalloc(ffb_plan_t p, const float *d_images, int64_t n, float *d_F, void *stream) {
    FFB_PLAN_HERE(p);
    if (!p || n < 0 || (n > 0 && (!d_images || !d_F))) return FFB_ERR_ARG;
    const int N = p->N, L = p->L, Nh = N / 2 + 1;
    const size_t h_bytes = (sizeof(float2) * (size_t)Nh * L + 255) / 256 * 256;
    const size_t g_bytes = (sizeof(float2) * (size_t)p->Mh * N + 255) / 256 * 256;
    const size_t per_image = h_bytes + g_bytes;
    if (per_image > FFB_NOALLOC_SCRATCH_BYTES) return FFB_ERR_UNSUPPORTED;  // one image does not fit
    if (n == 0) return FFB_OK;
    void *base = nullptr;
    int e = noalloc_scratch_address(&base);
    if (e) return e;
    const int group = (int)(FFB_NOALLOC_SCRATCH_BYTES / per_image);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sm_rows = sizeof(float2) * ((size_t)ROW_WARPS * 2 * N + (size_t)Nh * 2 * ROW_WARPS);
    const size_t sm_cols = sizeof(float2) * (size_t)COL_WARPS * 2 * N;
    if ((e = noalloc_smem((const void *)k_rows, sm_rows))) return e;
    if ((e = noalloc_smem((const void *)k_cols, sm_cols))) return e;
    const size_t per_out = (size_t)p->n_xi * (p->n_theta / 2) * 2;  // floats per image
    for (int64_t i0 = 0; i0 < n; i0 += group) {
        const int m = (int)((n - i0) < group ? (n - i0) : group);
        float2 *H = (float2 *)base;
        float2 *G = (float2 *)((unsigned char *)base + h_bytes * (size_t)m);
        dim3 g1((L + 2 * ROW_WARPS - 1) / (2 * ROW_WARPS), m);
        k_rows<<<g1, 32 * ROW_WARPS, sm_rows, s>>>(d_images + (size_t)i0 * L * L, L, p->off, N, p->d_corr,
                                                    p->d_twN, p->fftN, H, p->d_status);
        dim3 g2((Nh + COL_WARPS - 1) / COL_WARPS, m);
        k_cols<<<g2, 32 * COL_WARPS, sm_cols, s>>>(H, L, p->off, N, p->h, p->Mh, p->d_twN, p->fftN, G);
        dim3 g3((p->n_xi + RING_RB - 1) / RING_RB, m);
        k_interp_ring<true, RING_RB><<<g3, RING_NT, 0, s>>>(G, N, p->h, p->Mh, p->w, (float)p->beta, p->d_rad,
                                                            p->d_ang, p->n_xi, p->n_theta, p->d_twT, p->fftT,
                                                            p->k_max, m, nullptr,
                                                            (float2 *)(d_F + (size_t)i0 * per_out), p->d_status);
        p->launches += 3;
        e = ffb_check_cuda(cudaGetLastError());
        if (e) return e;
    }
    return FFB_OK;
}
