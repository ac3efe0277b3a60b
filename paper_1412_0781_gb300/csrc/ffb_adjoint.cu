// ffb_adjoint.cu -- the adjoint T y = Re(M^H y) of the expansion (step a10),
// built as the exact transpose of each forward step for the real inner
// products Re sum conj(u) v (complex vectors) and sum x y (images):
//
//   forward                                 adjoint (this file)
//   a = B Fhat, Im a_0 := 0                 Yhat = B^T y, Im y_0 := 0
//   Fhat_k = s DFT(ring)_k, k <= k_max,     g = inverse DFT of Yhat (zero-padded),
//     ring = [F_l, conj F_l] (l < n/2)       G_l = s (g_l + conj g_{l+n/2})
//   F_pt = sum psi psi Gext[tap]            Gext[tap] += psi psi G_pt (spreading; for
//                                            the fused path's plans in shared memory
//                                            per image half, ffb_grid.cu)
//   Gext = halo copy of G (conj mirror)     G += conj(mirror of the halo rows)
//   G[.][m2] = DFT over i1 of H[m2][.]      H[m2][a1] = inverse DFT over m1
//   H[m2][a1] = DFT over i2 (real rows)     P'[a1][i2] = Re sum_{m2=0}^{N/2} H e^{+...}
//   P' = I corr corr                        I* = P' corr corr
//
// s = 2 pi / n_theta.  Inverse DFTs carry the + sign and no 1/N factor.
#include "ffb_internal.cuh"

#define ADJ_RB 8
#define ADJ_NT 256
#define AROW_WARPS 8
#define ACOL_WARPS 8
#define ABES_IMG 32

// ---------------------------------------------------------------------------
// transposed radial quadrature: Yhat[k][img][c][j] = sum_q B_{kqj} y[img][o_k+q].c
// grid (ceil(nimg/32), k_max+1), 256 threads; thread owns 2 images x (re,im)
// x 4 j values per pass over j tiles of 64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_adj_bessel(const float2 *__restrict__ y, const float *__restrict__ Bf, const int *__restrict__ pk_,
             const int *__restrict__ off_, int n_xi, int chunk, int nimg, int P, float *__restrict__ Yhat) {
    extern __shared__ float smb[];
    const int k = blockIdx.y;
    const int pk = pk_[k], o = off_[k];
    const int i0 = blockIdx.x * ABES_IMG;
    const int ldq = pk + 1;
    float *Ys = smb;              // [64 rows (img, c)][ldq]
    float *Bs = smb + 64 * ldq;   // [64 j][ldq]   B^T tile: Bs[j][q]
    for (int t = threadIdx.x; t < ABES_IMG * pk; t += 256) {
        int ii = t / pk, q = t - ii * pk;
        float2 v = make_float2(0.f, 0.f);
        if (i0 + ii < nimg) v = __ldg(&y[(size_t)(i0 + ii) * P + o + q]);
        Ys[(2 * ii) * ldq + q] = v.x;
        Ys[(2 * ii + 1) * ldq + q] = (k == 0) ? 0.f : v.y;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int j0 = 0; j0 < n_xi; j0 += 64) {
        __syncthreads();
        for (int t = threadIdx.x; t < 64 * pk; t += 256) {
            int q = t >> 6, jj = t & 63;
            Bs[jj * ldq + q] = (j0 + jj < n_xi) ? __ldg(&Bf[(size_t)(o + q) * n_xi + j0 + jj]) : 0.f;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        for (int q = 0; q < pk; ++q) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = Ys[(ty * 4 + r) * ldq + q];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[(tx + 16 * c) * ldq + q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = ty * 4 + r;        // (image, c)
            const int img = i0 + row / 2, cc = row & 1;
            if (img >= nimg) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + tx + 16 * c;
                if (j < n_xi) Yhat[(((size_t)k * chunk + img) * 2 + cc) * n_xi + j] = acc[r][c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// inverse ring DFT + fold + spreading onto the extended half grid (zeroed
// beforehand).  grid (ceil(n_xi/RB), nimg), ADJ_NT threads,
// RB rings per CTA.
// ---------------------------------------------------------------------------
template <int RB>
__global__ void __launch_bounds__(ADJ_NT)
k_adj_ring_spread(const float *__restrict__ Yhat, int N, int h, int Mh, int w, float beta,
                  const float2 *__restrict__ rad, const float4 *__restrict__ ang, int n_xi, int n_theta,
                  const float2 *__restrict__ twT, FftPlanDev fpT, int kmax, int chunk,
                  float2 *__restrict__ Gext, int *status) {
    extern __shared__ float2 sm[];
    float2 *ringA = sm;
    float2 *ringB = sm + RB * n_theta;
    const int img = blockIdx.y;
    const int j0 = blockIdx.x * RB;
    const int nh = n_theta / 2;
    for (int t = threadIdx.x; t < RB * n_theta; t += ADJ_NT) ringA[t] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int t = threadIdx.x; t < (kmax + 1) * 2 * RB; t += ADJ_NT) {
        const int jj = t % RB, cc = (t / RB) & 1, k = t / (2 * RB);
        const int j = j0 + jj;
        if (j < n_xi) {
            float v = __ldg(&Yhat[(((size_t)k * chunk + img) * 2 + cc) * n_xi + j]);
            if (cc) ringA[jj * n_theta + k].y = v;
            else ringA[jj * n_theta + k].x = v;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int jj = warp; jj < RB; jj += ADJ_NT / 32)
        smem_fft<true>(ringA + jj * n_theta, ringB + jj * n_theta, fpT, twT, lane, 32, WarpSync());
    __syncthreads();
    const float2 *g = (fpT.nst & 1) ? ringB : ringA;
    const float scale = 6.283185307179586f / (float)n_theta;
    float2 *Gi = Gext + (size_t)img * Mh * N;
    const float halfw = 0.5f * (float)w;
    const float two_over_w = 2.0f / (float)w;
    for (int t = threadIdx.x; t < RB * nh; t += ADJ_NT) {
        const int jj = t / nh, l = t - jj * nh;
        const int j = j0 + jj;
        if (j >= n_xi) continue;
        float2 a = g[jj * n_theta + l], b = g[jj * n_theta + l + nh];
        float2 val = make_float2(scale * (a.x + b.x), scale * (a.y - b.y));
        const float2 r = __ldg(&rad[j]);
        const float4 an = __ldg(&ang[l]);
        float p1 = r.x * an.x;
        float e1 = fmaf(r.x, an.x, -p1) + fmaf(r.x, an.y, r.y * an.x);
        float p2 = r.x * an.z;
        float e2 = fmaf(r.x, an.z, -p2) + fmaf(r.x, an.w, r.y * an.z);
        float m1f = ceilf(p1 - halfw), m2f = ceilf(p2 - halfw);
        float f1 = (p1 - m1f) + e1, f2 = (p2 - m2f) + e2;
        int m1 = (int)m1f, m2 = (int)m2f;
        if (m2 + h < 0 || m2 + w - 1 + h >= Mh || m1 < -N || m1 > N) {
            ffb_flag(status, FFB_ERR_ARG);
            continue;
        }
        float wx[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q < w) wx[q] = es_kernel(f1 - (float)q, two_over_w, beta);
        for (int bb = 0; bb < w; ++bb) {
            const float wy = es_kernel(f2 - (float)bb, two_over_w, beta);
            float2 *row = Gi + (size_t)(m2 + bb + h) * N;
            const float2 vy = make_float2(wy * val.x, wy * val.y);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (q < w) {
                    int mm = m1 + q;
                    if (mm < 0) mm += N;
                    else if (mm >= N) mm -= N;
                    atomicAdd(&row[mm], make_float2(wx[q] * vy.x, wx[q] * vy.y));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// inverse ring DFT + fold only (fused-path plans, whose spreading runs in
// ffb_grid.cu): Gpol[img][j][l] = s (g_l + conj g_{l + n/2}), l < n/2, the
// layout of the forward's polar buffer.  grid (ceil(n_xi/RB), nimg).
// ---------------------------------------------------------------------------
template <int RB>
__global__ void __launch_bounds__(ADJ_NT)
k_adj_ring_polar(const float *__restrict__ Yhat, int n_xi, int n_theta, const float2 *__restrict__ twT,
                 FftPlanDev fpT, int kmax, int chunk, float2 *__restrict__ Gpol) {
    extern __shared__ float2 sm[];
    float2 *ringA = sm;
    float2 *ringB = sm + RB * n_theta;
    const int img = blockIdx.y;
    const int j0 = blockIdx.x * RB;
    const int nh = n_theta / 2;
    for (int t = threadIdx.x; t < RB * n_theta; t += ADJ_NT) ringA[t] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int t = threadIdx.x; t < (kmax + 1) * 2 * RB; t += ADJ_NT) {
        const int jj = t % RB, cc = (t / RB) & 1, k = t / (2 * RB);
        const int j = j0 + jj;
        if (j < n_xi) {
            float v = __ldg(&Yhat[(((size_t)k * chunk + img) * 2 + cc) * n_xi + j]);
            if (cc) ringA[jj * n_theta + k].y = v;
            else ringA[jj * n_theta + k].x = v;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int jj = warp; jj < RB; jj += ADJ_NT / 32)
        smem_fft<true>(ringA + jj * n_theta, ringB + jj * n_theta, fpT, twT, lane, 32, WarpSync());
    __syncthreads();
    const float2 *g = (fpT.nst & 1) ? ringB : ringA;
    const float scale = 6.283185307179586f / (float)n_theta;
    float2 *Gi = Gpol + (size_t)img * n_xi * nh;
    for (int t = threadIdx.x; t < RB * nh; t += ADJ_NT) {
        const int jj = t / nh, l = t - jj * nh;
        const int j = j0 + jj;
        if (j >= n_xi) continue;
        const float2 a = g[jj * n_theta + l], b = g[jj * n_theta + l + nh];
        Gi[(size_t)j * nh + l] = make_float2(scale * (a.x + b.x), scale * (a.y - b.y));
    }
}

// ---------------------------------------------------------------------------
// halo fold + inverse column DFT: for column m2 in [0, N/2],
// Gc[m1] = Gext[m2+h][m1] (+ conj Gext[h-m2][-m1] if 1 <= m2 <= h)
//                         (+ conj Gext[h+N-m2][-m1] if N/2-h <= m2 <= N/2-1);
// H[m2][a1] = sum_m1 Gc[m1] e^{+2 pi i m1 (a1-off)/N}.
// grid (ceil((N/2+1)/ACOL_WARPS), nimg)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * ACOL_WARPS)
k_adj_cols(const float2 *__restrict__ Gext, int L, int off, int N, int h, int Mh,
           const float2 *__restrict__ tw, FftPlanDev fp, float2 *__restrict__ H) {
    extern __shared__ float2 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int img = blockIdx.y;
    const int Nh = N / 2 + 1;
    const int m2 = blockIdx.x * ACOL_WARPS + warp;
    if (m2 >= Nh) return;
    float2 *bufA = sm + warp * 2 * N;
    float2 *bufB = bufA + N;
    const float2 *Gi = Gext + (size_t)img * Mh * N;
    const float2 *row = Gi + (size_t)(m2 + h) * N;
    const bool lo = (m2 >= 1 && m2 <= h);
    const bool hi = (m2 >= 1 && m2 >= N / 2 - h && m2 <= N / 2 - 1);
    const float2 *rlo = Gi + (size_t)(h - m2) * N;
    const float2 *rhi = Gi + (size_t)(h + N - m2) * N;
    for (int m1 = lane; m1 < N; m1 += 32) {
        float2 v = row[m1];
        const int mr = (m1 == 0) ? 0 : N - m1;
        if (lo) v = cadd(v, cconj(rlo[mr]));
        if (hi) v = cadd(v, cconj(rhi[mr]));
        bufA[m1] = v;
    }
    __syncwarp();
    float2 *X = smem_fft<true>(bufA, bufB, fp, tw, lane, 32, WarpSync());
    float2 *Hc = H + ((size_t)img * Nh + m2) * L;
    for (int a1 = lane; a1 < L; a1 += 32) {
        int pos = a1 - off;
        if (pos < 0) pos += N;
        Hc[a1] = X[pos];
    }
}

// ---------------------------------------------------------------------------
// rows: I*[a1][a2] = corr[a1] corr[a2] Re sum_{m2=0}^{N/2} H[m2][a1]
// e^{+2 pi i m2 (a2-off)/N}, two rows per complex inverse FFT through the
// Hermitian symmetrisation Y_s[m] = (Y[m] + conj Y[N-m]) / 2 (Y = 0 beyond N/2).
// grid (ceil(L / 2 AROW_WARPS), nimg)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * AROW_WARPS)
k_adj_rows(const float2 *__restrict__ H, int L, int off, int N, const float *__restrict__ corr,
           const float2 *__restrict__ tw, FftPlanDev fp, float *__restrict__ out) {
    extern __shared__ float2 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int img = blockIdx.y;
    const int a1 = blockIdx.x * 2 * AROW_WARPS + 2 * warp;
    const int Nh = N / 2 + 1;
    if (a1 >= L) return;
    const bool two = (a1 + 1) < L;
    float2 *bufA = sm + warp * 2 * N;
    float2 *bufB = bufA + N;
    const float2 *Hi = H + (size_t)img * Nh * L;
    for (int m = lane; m < N; m += 32) {
        // Y_a[m] (m <= N/2) and the mirrored conj Y_a[N-m]
        float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
        if (m < Nh) {
            ya = Hi[(size_t)m * L + a1];
            if (two) yb = Hi[(size_t)m * L + a1 + 1];
        }
        const int mr = (m == 0) ? 0 : N - m;
        float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
        if (mr < Nh) {
            ra = cconj(Hi[(size_t)mr * L + a1]);
            if (two) rb = cconj(Hi[(size_t)mr * L + a1 + 1]);
        }
        float2 sa = make_float2(0.5f * (ya.x + ra.x), 0.5f * (ya.y + ra.y));  // Hermitian
        float2 sb = make_float2(0.5f * (yb.x + rb.x), 0.5f * (yb.y + rb.y));
        bufA[m] = make_float2(sa.x - sb.y, sa.y + sb.x);                        // sa + i sb
    }
    __syncwarp();
    float2 *X = smem_fft<true>(bufA, bufB, fp, tw, lane, 32, WarpSync());
    const float c1 = corr[a1];
    const float c2 = two ? corr[a1 + 1] : 0.f;
    float *o1 = out + ((size_t)img * L + a1) * L;
    for (int a2 = lane; a2 < L; a2 += 32) {
        int pos = a2 - off;
        if (pos < 0) pos += N;
        float2 v = X[pos];
        const float ca = corr[a2];
        o1[a2] = v.x * c1 * ca;
        if (two) o1[L + a2] = v.y * c2 * ca;
    }
}

// ---------------------------------------------------------------------------
// chunked driver
// ---------------------------------------------------------------------------
static int set_smem(const void *fn, size_t bytes, int *cache) {
    if (bytes > 48 * 1024 && *cache < (int)bytes) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        if (e) return e;
        *cache = (int)bytes;
    }
    return FFB_OK;
}

int ffb_launch_adjoint(ffb_plan_t p, const float *d_coef, int64_t n, float *d_images, cudaStream_t s) {
    int e = ffb_ensure_scratch(p);
    if (e) return e;
    if ((e = ffb_ensure_scratch_grid(p))) return e;
    const int N = p->N, L = p->L, Nh = N / 2 + 1;
    static int a_bes = 0, a_ring = 0, a_ring4 = 0, a_ringp = 0, a_cols = 0, a_rows = 0;
    // ADJ_RB rings per CTA, or half as many where their ring buffers would
    // not fit in shared memory (n_theta > 1816 at 227 KB)
    const int rb = ffb_ring_buffers_fit(p->n_theta, ADJ_RB) ? ADJ_RB : ADJ_RB / 2;
    if (!ffb_ring_buffers_fit(p->n_theta, rb) || (p->fused && rb != ADJ_RB)) return FFB_ERR_UNSUPPORTED;
    const size_t sm_bes = sizeof(float) * 2 * 64 * (size_t)(p->pmax + 1);
    const size_t sm_ring = sizeof(float2) * 2 * rb * (size_t)p->n_theta;
    const size_t sm_cols = sizeof(float2) * (size_t)ACOL_WARPS * 2 * N;
    const size_t sm_rows = sizeof(float2) * (size_t)AROW_WARPS * 2 * N;
    static int a_ringp4 = 0;
    // plans with a polar buffer and a spreading table (fused path, tiled
    // separate-kernel path): inverse ring DFT to the polar buffer, then the
    // spreading in shared memory
    const bool polar = p->fused || p->ntblk > 0;
    if ((e = set_smem((const void *)k_adj_bessel, sm_bes, &a_bes))) return e;
    if (polar && rb == ADJ_RB) {
        if ((e = set_smem((const void *)k_adj_ring_polar<ADJ_RB>, sm_ring, &a_ringp))) return e;
    } else if (polar) {
        if ((e = set_smem((const void *)k_adj_ring_polar<ADJ_RB / 2>, sm_ring, &a_ringp4))) return e;
    } else if (rb == ADJ_RB) {
        if ((e = set_smem((const void *)k_adj_ring_spread<ADJ_RB>, sm_ring, &a_ring))) return e;
    } else {
        if ((e = set_smem((const void *)k_adj_ring_spread<ADJ_RB / 2>, sm_ring, &a_ring4))) return e;
    }
    if ((e = set_smem((const void *)k_adj_cols, sm_cols, &a_cols))) return e;
    if ((e = set_smem((const void *)k_adj_rows, sm_rows, &a_rows))) return e;
    for (int64_t i0 = 0; i0 < n; i0 += p->chunk) {
        const int m = (int)((n - i0) < p->chunk ? (n - i0) : p->chunk);
        {
            ProfScope ps(p, FFB_KC_ADJ_BESSEL, s);
            dim3 g((m + ABES_IMG - 1) / ABES_IMG, p->k_max + 1);
            k_adj_bessel<<<g, 256, sm_bes, s>>>((const float2 *)d_coef + (size_t)i0 * p->P, p->d_Bf, p->d_p,
                                                p->d_off, p->n_xi, p->chunk, m, p->P, p->d_Fhat);
            p->launches++;
        }
        e = ffb_check_cuda(cudaMemsetAsync(p->d_G, 0, sizeof(float2) * (size_t)m * p->Mh * N, s));
        if (e) return e;
        if (polar) {
            // inverse ring DFT to the polar buffer, then the half grids in
            // shared memory with the forward's unit or tile table
            if (p->ring_direct) {
                // register four-step inverse ring DFT (ffb_ring.cu)
                if ((e = ffb_launch_ring_ifft(p, m, p->d_Fhat, p->d_Fpol, s))) return e;
            } else {
                ProfScope ps(p, FFB_KC_ADJ_RING, s);
                dim3 g((p->n_xi + rb - 1) / rb, m);
                if (rb == ADJ_RB)
                    k_adj_ring_polar<ADJ_RB><<<g, ADJ_NT, sm_ring, s>>>(p->d_Fhat, p->n_xi, p->n_theta, p->d_twT,
                                                                        p->fftT, p->k_max, p->chunk, p->d_Fpol);
                else
                    k_adj_ring_polar<ADJ_RB / 2><<<g, ADJ_NT, sm_ring, s>>>(p->d_Fhat, p->n_xi, p->n_theta,
                                                                            p->d_twT, p->fftT, p->k_max,
                                                                            p->chunk, p->d_Fpol);
                p->launches++;
                if ((e = ffb_check_cuda(cudaGetLastError()))) return e;
            }
            if (p->fused) {
                if ((e = ffb_launch_fused_spread(p, p->d_Fpol, m, p->d_G, s))) return e;
            } else if ((e = ffb_launch_tile_spread(p, m, p->d_Fpol, p->d_G, s))) {
                return e;
            }
        } else {
            ProfScope ps(p, FFB_KC_ADJ_RING, s);
            dim3 g((p->n_xi + rb - 1) / rb, m);
            if (rb == ADJ_RB)
                k_adj_ring_spread<ADJ_RB><<<g, ADJ_NT, sm_ring, s>>>(
                    p->d_Fhat, N, p->h, p->Mh, p->w, (float)p->beta, p->d_rad, p->d_ang, p->n_xi, p->n_theta,
                    p->d_twT, p->fftT, p->k_max, p->chunk, p->d_G, p->d_status);
            else
                k_adj_ring_spread<ADJ_RB / 2><<<g, ADJ_NT, sm_ring, s>>>(
                    p->d_Fhat, N, p->h, p->Mh, p->w, (float)p->beta, p->d_rad, p->d_ang, p->n_xi, p->n_theta,
                    p->d_twT, p->fftT, p->k_max, p->chunk, p->d_G, p->d_status);
            p->launches++;
        }
        {
            ProfScope ps(p, FFB_KC_ADJ_COLS, s);
            dim3 g((Nh + ACOL_WARPS - 1) / ACOL_WARPS, m);
            k_adj_cols<<<g, 32 * ACOL_WARPS, sm_cols, s>>>(p->d_G, L, p->off, N, p->h, p->Mh, p->d_twN, p->fftN,
                                                           p->d_H);
            p->launches++;
        }
        {
            ProfScope ps(p, FFB_KC_ADJ_ROWS, s);
            dim3 g((L + 2 * AROW_WARPS - 1) / (2 * AROW_WARPS), m);
            k_adj_rows<<<g, 32 * AROW_WARPS, sm_rows, s>>>(p->d_H, L, p->off, N, p->d_corr, p->d_twN, p->fftN,
                                                           d_images + (size_t)i0 * L * L);
            p->launches++;
        }
        e = ffb_check_cuda(cudaGetLastError());
        if (e) return e;
    }
    return FFB_OK;
}
