// ffb_ring.cu -- step a4: the angular FFT of every ring of the polar samples
// (Eq. 1DFFT), written in the operand format of the radial quadrature.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ffb_fft.cuh"

// rings per ring-FFT CTA (one warp each): 32; 16 at n_theta = 512, where two
// such CTAs share an SM and their barrier waits overlap (32 rings: one CTA
// per SM, 18.3 ms per 100k images at L = 128; 16: 16.9 ms; 8: 18.5 ms); 8 at
// n_theta = 1024, where a warp's transpose buffer holds 32 x 32 values
#ifndef FFB_RFFT_RB512
#define FFB_RFFT_RB512 16
#endif
template <int NTH>
constexpr int rfft_rb() { return NTH > 512 ? 8 : (NTH == 512 ? FFB_RFFT_RB512 : 32); }
// CTAs per SM the register budget aims at (n_theta <= 512: 32 warps per SM
// at 64 registers, whatever the rings per CTA)
template <int NTH, int RB>
constexpr int rfft_minb() { return NTH <= 512 ? 32 / RB : 1; }

// cos / sin (2 pi m / M) for M = 2 .. 32
template <int M>
__device__ __forceinline__ float wcos(int m) { return (M <= 16) ? cos16((16 / (M <= 16 ? M : 16)) * m) : cos32(m); }
template <int M>
__device__ __forceinline__ float wsin(int m) { return (M <= 16) ? sin16((16 / (M <= 16 ? M : 16)) * m) : sin32(m); }

// ---------------------------------------------------------------------------
// ring FFT: F[img][j][l] (l < n_theta/2) -> Fhat[k][img][c][j], k <= k_max,
// with the conjugate completion of the ring and the 2 pi / n_theta weight.
//
// One warp per ring, four-step in registers: with n_theta = 32 M (M <= 32), sample
// l = 32 m + j (lane j) and k = k1 + M k2,
//   X_k = sum_j W^{j k1} [sum_m s_{32m+j} W_M^{m k1}] W_32^{j k2},  W = e^{-2 pi i / n_theta}.
// Pass A: each lane loads its M/2 samples x_m (m < M/2) from the polar
// buffer; with s_{l + n_theta/2} = conj s_l the length-M DFT over m splits
// into X[2j] = 2 DFT_{M/2}(Re x_m)[j] (a real-input DFT) and X[2j+1] =
// 2 DFT_{M/2}(i Im(x_m) W_M^m)[j] (the factor 2 goes into the weight); then
// the twiddle W^{j k1}.  A transpose through
// shared memory (row k1, column rotated by k1 R, R = 32/M, so that writes and
// reads touch 16 distinct bank slots per half warp) gives lane (g = k1, r) the
// values j = r + R i.  Pass B: the length-32 DFT over j for every k1 as a
// length-M DFT over i in registers, the twiddle W_32^{r k2'} and a length-R
// DFT across the R lanes of the group (radix-2 decimation in frequency by XOR
// shuffles; lane r ends with t = bitreverse(r)), k2 = k2' + M t.  For
// n_theta = 512 (R = 2) the twiddles are constants and, as k_max < n_theta/2,
// only the t = 0 half of the last step is formed (the pair's sum).  The
// results with k <= k_max go to a ring-major shared stage and leave as rows
// of RFFT_RB consecutive rings per (k, re/im) in the quadrature's operand
// format, two rings per store.
// grid (ceil(n_xi / RFFT_RB), nimg), 32 RFFT_RB threads.
// ---------------------------------------------------------------------------
template <int NTH, int FMT, int RFFT_RB = rfft_rb<NTH>()>
__global__ void __launch_bounds__(32 * RFFT_RB, rfft_minb<NTH, RFFT_RB>())
k_ring_fft(const float2 *__restrict__ Fpol, int n_xi, int kmax, int lead, const float2 *__restrict__ twT,
           const float2 *__restrict__ twA,
           void *__restrict__ out0, void *__restrict__ out1, int ld) {
    constexpr int M = NTH / 32;      // samples per lane
    constexpr int R = 32 / M;        // lanes per length-32 DFT of pass B
    constexpr int NH = NTH / 2;
    static_assert(M >= 2 && M <= 32 && M * R == 32, "n_theta in {64, 128, 256, 512, 1024}");
    extern __shared__ float2 smr[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *tb = smr + warp * (M * 32);                  // this warp's transpose buffer [M][32]
    float *ost = (float *)(smr + RFFT_RB * M * 32);      // [RFFT_RB][ostld]: ring-major stage
    const int ostld = (2 * (kmax + 1)) | 1;              // odd: the write-out reads conflict-free
    const int img = blockIdx.y;
    const int j0 = blockIdx.x * RFFT_RB;
    pdl_trigger();
    pdl_wait();   // the polar buffer comes from the previous kernel
    const int ring = j0 + warp;
    // pass A below yields half of each DFT value: the weight 2 pi / n_theta
    // carries the factor 2
    const float scale = 2.f * 6.283185307179586f / (float)NTH;
    if (ring < n_xi) {
        const float2 *src = Fpol + ((size_t)img * n_xi + ring) * NH;
        // pass A over m with s_{l + n_theta/2} = conj s_l: for the M/2 loaded
        // samples x_m, X[2j] / 2 is the length-M/2 DFT of Re x_m and
        // X[2j+1] / 2 that of i Im(x_m) W_M^m
        float u[M / 2];
        float2 v[M / 2], E[M / 2];
#pragma unroll
        for (int m = 0; m < M / 2; ++m) {
            // read once: evict first, so that the planes stay in L2 longer
            const float2 xm = ldg_hint(&src[32 * m + lane], l2_evict_first());
            u[m] = xm.x;
            v[m] = make_float2(xm.y * wsin<M>(m), xm.y * wcos<M>(m));
        }
        dft_real<M / 2>(u, E);
        dft_reg<M / 2>(v);
        float2 x[M];
#pragma unroll
        for (int j = 0; j < M / 2; ++j) {
            x[2 * j] = E[j];
            x[2 * j + 1] = v[j];
        }
        // twiddles W^{j k1} from the plan's table [k1][j] (coalesced)
#pragma unroll
        for (int k1 = 1; k1 < M; ++k1) x[k1] = cmul(x[k1], __ldg(&twA[k1 * 32 + lane]));
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) tb[k1 * 32 + ((lane + k1 * R) & 31)] = x[k1];
        __syncwarp();
        const int g = lane / R, r = lane % R;
        float2 y[M];
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = tb[g * 32 + ((r + R * i + g * R) & 31)];
        dft_reg<M>(y);                         // pass B, part 1: over i
        float *row = ost + warp * ostld;
        if constexpr (R == 2) {
            // twiddle W_32^{r k2} (constants), then only the half k < n_theta/2
            // of the last radix-2 step (k_max < n_theta/2): the pair's sum, of
            // which lane r keeps the outputs k2 in [r M/2, (r + 1) M/2)
#pragma unroll
            for (int k2 = 1; k2 < M; ++k2) {
                const float2 w = make_float2(cos32(k2), -sin32(k2));
                const float2 t = cmul(y[k2], w);
                y[k2] = r ? t : y[k2];
            }
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                y[k2].x += __shfl_xor_sync(0xffffffffu, y[k2].x, 1);
                y[k2].y += __shfl_xor_sync(0xffffffffu, y[k2].y, 1);
            }
            // the two lanes of a pair write the same bank slot for their k:
            // one takes the real part first, the other the imaginary part
#pragma unroll
            for (int h2 = 0; h2 < M / 2; ++h2) {
                const float2 val = r ? y[M / 2 + h2] : y[h2];
                const int k = g + M * (r * (M / 2) + h2);
                if (k <= kmax) {
                    row[2 * k + r] = scale * (r ? val.y : val.x);
                    row[2 * k + 1 - r] = scale * (r ? val.x : val.y);
                }
            }
        } else if constexpr (R == 1) {
            // one lane per k1: the length-32 DFT over i gave k = g + 32 k2
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int k = g + M * k2;
                if (k <= kmax) {
                    row[2 * k] = scale * y[k2].x;
                    row[2 * k + 1] = scale * y[k2].y;
                }
            }
        } else {
#pragma unroll
            for (int k2 = 1; k2 < M; ++k2) y[k2] = cmul(y[k2], __ldg(&twT[(r * k2 * (NTH / 32)) & (NTH - 1)]));
#pragma unroll
            for (int h = R / 2; h >= 1; h >>= 1) {           // pass B, part 2: across the R lanes
                const bool up = (r & h) != 0;
                // the last stage (h = 1) has the twiddle W^0 = 1
                const float2 w = (h > 1) ? __ldg(&twT[(r & (h - 1)) * (NTH / (2 * h))]) : make_float2(1.f, 0.f);
#pragma unroll
                for (int k2 = 0; k2 < M; ++k2) {
                    const float2 pv = make_float2(__shfl_xor_sync(0xffffffffu, y[k2].x, h),
                                                  __shfl_xor_sync(0xffffffffu, y[k2].y, h));
                    const float2 d = csub(pv, y[k2]);
                    y[k2] = up ? ((h > 1) ? cmul(d, w) : d) : cadd(y[k2], pv);
                }
            }
            int t = 0;
            for (int b = 1; b < R; b <<= 1) t = (t << 1) | ((r & b) ? 1 : 0);
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int k = g + M * (k2 + M * t);
                if (k <= kmax) {
                    row[2 * k] = scale * y[k2].x;
                    row[2 * k + 1] = scale * y[k2].y;
                }
            }
        }
    }
    __syncthreads();
    // write-out: thread t owns the ring pair jj = 2 (t % (RFFT_RB / 2)), jj + 1
    // and the (k, re/im) rows kc = t / (RFFT_RB / 2) + KCSTEP it; KCSTEP is
    // even, so re/im of a row is fixed per thread; the pair leaves as one
    // 2-element store per plane
    const int nr = min(RFFT_RB, n_xi - j0);
    constexpr int NPR = RFFT_RB / 2;
    constexpr int KCSTEP = (32 * RFFT_RB) / NPR;
    static_assert(KCSTEP % 2 == 0, "re/im fixed per thread");
    const int jj = 2 * (threadIdx.x % NPR);
    const int kc0 = threadIdx.x / NPR;
    const int kcend = 2 * (kmax + 1);
    if (jj < nr) {
        const bool two = jj + 1 < nr;
        size_t idx = (((size_t)(kc0 >> 1) * lead + img) * 2 + (kc0 & 1)) * ld + j0 + jj;
        const size_t step = (size_t)(KCSTEP / 2) * lead * 2 * ld;
        for (int kc = kc0; kc < kcend; kc += KCSTEP, idx += step) {
            const float x0 = ost[jj * ostld + kc];
            const float x1 = two ? ost[(jj + 1) * ostld + kc] : 0.f;
            if (FMT == FFB_FMT_F32) {
                if (two) *(float2 *)((float *)out0 + idx) = make_float2(x0, x1);
                else ((float *)out0)[idx] = x0;
            } else if (FMT == FFB_FMT_TF32 || FMT == FFB_FMT_TF32X2) {
                const float h0 = tf32_round(x0), h1 = tf32_round(x1);
                if (two) {
                    *(float2 *)((float *)out0 + idx) = make_float2(h0, h1);
                    if (FMT == FFB_FMT_TF32X2) *(float2 *)((float *)out1 + idx) = make_float2(x0 - h0, x1 - h1);
                } else {
                    ((float *)out0)[idx] = h0;
                    if (FMT == FFB_FMT_TF32X2) ((float *)out1)[idx] = x0 - h0;
                }
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                if (two) {
                    // the quadrature reads the planes later in the step: evict last
                    const unsigned long long pl = l2_evict_last();
                    st_hint((__nv_bfloat16 *)out0 + idx, *(const unsigned *)&h, pl);
                    if (FMT == FFB_FMT_BF16X2) st_hint((__nv_bfloat16 *)out1 + idx, *(const unsigned *)&l, pl);
                } else {
                    ((__nv_bfloat16 *)out0)[idx] = __low2bfloat16(h);
                    if (FMT == FFB_FMT_BF16X2) ((__nv_bfloat16 *)out1)[idx] = __low2bfloat16(l);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse ring DFT of the adjoint (step a10, the transpose of Eq. 1DFFT with
// the ring's conjugate completion): from the ring spectra Y_k, k <= k_max
// (Yhat[k][img][c][j], float32, from the transposed quadrature), the polar
// values G_l = s (g_l + conj g_{l + n/2}), l < n/2, of the zero-padded
// inverse DFT g_l = sum_k Y_k e^{+2 pi i k l / n}, s = 2 pi / n.  Written out,
//   G_l = s sum_k [Y_k e^{+i theta_l k} + (-1)^k conj(Y_k) e^{-i theta_l k}]
//       = s conj( DFT_n(W)_l ),
// W_0 = 2 Re Y_0, W_k = conj Y_k and W_{n-k} = (-1)^k Y_k for 1 <= k <= k_max,
// zero elsewhere.  The forward DFT of W is the four-step of k_ring_fft with a
// full length-M first pass (W has no symmetry); the outputs l < n/2 are the
// t = 0 half.  A CTA stages its rings' Y into shared memory (coalesced over
// rings), each warp forms its ring's W, transforms it, and the ring's
// results leave as one contiguous run of n/2 values of the polar buffer.
// grid (ceil(n_xi / RFFT_RB), nimg), 32 RFFT_RB threads.
// ---------------------------------------------------------------------------
template <int NTH, int RFFT_RB = rfft_rb<NTH>()>
__global__ void __launch_bounds__(32 * RFFT_RB, 1)
k_ring_ifft(const float *__restrict__ Yhat, int n_xi, int kmax, int chunk, const float2 *__restrict__ twT,
            const float2 *__restrict__ twA, float2 *__restrict__ Gpol) {
    constexpr int M = NTH / 32;
    constexpr int R = 32 / M;
    constexpr int NH = NTH / 2;
    constexpr int PR = NH + 1;       // pitch of a ring's region (odd in 8-byte slots)
    static_assert(M >= 2 && M <= 32 && M * R == 32, "n_theta in {64, 128, 256, 512, 1024}");
    extern __shared__ float2 smr[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *tb = smr + warp * (M * 32);                  // this warp's transpose buffer [M][32]
    float2 *region = smr + RFFT_RB * M * 32;             // [RFFT_RB][PR]: Y_k, then G_l
    const int img = blockIdx.y;
    const int j0 = blockIdx.x * RFFT_RB;
    // Y_k of the CTA's rings: thread t takes (k, ring) = (t / RB, t % RB), the
    // re and im rows of Yhat coalesced over rings
    for (int t = threadIdx.x; t < (kmax + 1) * RFFT_RB; t += 32 * RFFT_RB) {
        const int k = t / RFFT_RB, jj = t - k * RFFT_RB;
        float2 v = make_float2(0.f, 0.f);
        if (j0 + jj < n_xi) {
            const size_t b = (((size_t)k * chunk + img) * 2) * n_xi + j0 + jj;
            v = make_float2(__ldg(&Yhat[b]), __ldg(&Yhat[b + n_xi]));
        }
        region[jj * PR + k] = v;
    }
    __syncthreads();
    const int ring = j0 + warp;
    if (ring >= n_xi) return;            // no block-wide barrier below
    float2 *reg = region + warp * PR;
    // W at w = 32 m + lane
    float2 x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int w = 32 * m + lane;
        float2 v = make_float2(0.f, 0.f);
        if (w == 0) {
            v = make_float2(2.f * reg[0].x, 0.f);
        } else if (w <= kmax) {
            v = cconj(reg[w]);
        } else if (w >= NTH - kmax) {
            const int k = NTH - w;
            v = reg[k];
            if (k & 1) v = make_float2(-v.x, -v.y);
        }
        x[m] = v;
    }
    dft_reg<M>(x);                                       // pass A: over m
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) x[k1] = cmul(x[k1], __ldg(&twA[k1 * 32 + lane]));
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) tb[k1 * 32 + ((lane + k1 * R) & 31)] = x[k1];
    __syncwarp();
    const int g = lane / R, r = lane % R;
    float2 y[M];
#pragma unroll
    for (int i = 0; i < M; ++i) y[i] = tb[g * 32 + ((r + R * i + g * R) & 31)];
    dft_reg<M>(y);                                       // pass B, part 1: over i
    const float scale = 6.283185307179586f / (float)NTH;
    // every lane has read its W above and the transpose is past a warp
    // barrier: the region now takes the results
    if constexpr (R == 1) {
#pragma unroll
        for (int k2 = 0; k2 < M / 2; ++k2) {
            const int l = g + M * k2;
            reg[l] = make_float2(scale * y[k2].x, -scale * y[k2].y);
        }
    } else if constexpr (R == 2) {
#pragma unroll
        for (int k2 = 1; k2 < M; ++k2) {
            const float2 w = make_float2(cos32(k2), -sin32(k2));
            const float2 t = cmul(y[k2], w);
            y[k2] = r ? t : y[k2];
        }
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            y[k2].x += __shfl_xor_sync(0xffffffffu, y[k2].x, 1);
            y[k2].y += __shfl_xor_sync(0xffffffffu, y[k2].y, 1);
        }
#pragma unroll
        for (int h2 = 0; h2 < M / 2; ++h2) {
            const int k2 = r * (M / 2) + h2;
            const float2 val = r ? y[M / 2 + h2] : y[h2];
            reg[g + M * k2] = make_float2(scale * val.x, -scale * val.y);
        }
    } else {
#pragma unroll
        for (int k2 = 1; k2 < M; ++k2) y[k2] = cmul(y[k2], __ldg(&twT[(r * k2 * (NTH / 32)) & (NTH - 1)]));
#pragma unroll
        for (int h = R / 2; h >= 1; h >>= 1) {
            const bool up = (r & h) != 0;
            const float2 w = (h > 1) ? __ldg(&twT[(r & (h - 1)) * (NTH / (2 * h))]) : make_float2(1.f, 0.f);
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const float2 pv = make_float2(__shfl_xor_sync(0xffffffffu, y[k2].x, h),
                                              __shfl_xor_sync(0xffffffffu, y[k2].y, h));
                const float2 d = csub(pv, y[k2]);
                y[k2] = up ? ((h > 1) ? cmul(d, w) : d) : cadd(y[k2], pv);
            }
        }
        int t = 0;
        for (int b = 1; b < R; b <<= 1) t = (t << 1) | ((r & b) ? 1 : 0);
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            const int l = g + M * (k2 + M * t);
            if (l < NH) reg[l] = make_float2(scale * y[k2].x, -scale * y[k2].y);
        }
    }
    __syncwarp();
    float2 *dst = Gpol + ((size_t)img * n_xi + ring) * NH;
    for (int l = lane; l < NH; l += 32) dst[l] = reg[l];
}

template <int NTH>
static int launch_ring_ifft(ffb_plan_t p, int m, const float *Yhat, float2 *Gpol, cudaStream_t s) {
    constexpr int RB = rfft_rb<NTH>();
    static int attr = 0;
    const size_t smem = sizeof(float2) * (size_t)RB * (NTH + NTH / 2 + 1);
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_ring_ifft<NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((p->n_xi + RB - 1) / RB, m);
    ProfScope ps(p, FFB_KC_ADJ_RING, s);
    k_ring_ifft<NTH><<<g, 32 * RB, smem, s>>>(Yhat, p->n_xi, p->k_max, p->chunk, (const float2 *)p->d_twT,
                                               (const float2 *)p->d_twA, Gpol);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// the adjoint's inverse ring DFT for plans whose ring FFT runs in registers
int ffb_launch_ring_ifft(ffb_plan_t p, int m, const float *Yhat, float2 *Gpol, cudaStream_t s) {
    if (p->k_max >= p->n_theta / 2) return FFB_ERR_UNSUPPORTED;
    switch (p->n_theta) {
        case 64: return launch_ring_ifft<64>(p, m, Yhat, Gpol, s);
        case 128: return launch_ring_ifft<128>(p, m, Yhat, Gpol, s);
        case 256: return launch_ring_ifft<256>(p, m, Yhat, Gpol, s);
        case 512: return launch_ring_ifft<512>(p, m, Yhat, Gpol, s);
        case 1024: return launch_ring_ifft<1024>(p, m, Yhat, Gpol, s);
        default: return FFB_ERR_UNSUPPORTED;
    }
}

// ring FFT twiddles of the plan (built with the fused path's tables)
int ffb_ring_prepare(ffb_plan_t p, cudaStream_t s) {
    int e = FFB_OK;
    // twiddles W^{j k1}, W = e^{-2 pi i / n_theta}, as [k1][j]
    // (k1 < n_theta / 32, j < 32), from float64
    const int MA = p->n_theta / 32;
    std::vector<float2> twa((size_t)MA * 32);
    for (int k1 = 0; k1 < MA; ++k1)
        for (int j = 0; j < 32; ++j) {
            const double a = -2.0 * M_PI * (double)((j * k1) % p->n_theta) / (double)p->n_theta;
            twa[(size_t)k1 * 32 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    if (p->d_twA) cudaFree(p->d_twA);
    p->d_twA = nullptr;
    e = ffb_check_cuda(cudaMalloc((void **)&p->d_twA, sizeof(float2) * twa.size()));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_twA, twa.data(), sizeof(float2) * twa.size(),
                                               cudaMemcpyHostToDevice, s));
    if (e) return e;
    return ffb_check_cuda(cudaStreamSynchronize(s));
}

template <int NTH, int FMT>
static int launch_ring_fmt(ffb_plan_t p, int m, const float2 *Fpol, const RingOut &o, cudaStream_t s) {
    constexpr int RFFT_RB = rfft_rb<NTH>();
    static int attr = 0;
    const size_t smem = sizeof(float2) * RFFT_RB * (size_t)NTH + sizeof(float) * RFFT_RB * ((2 * (p->k_max + 1)) | 1);
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_ring_fft<NTH, FMT>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((p->n_xi + RFFT_RB - 1) / RFFT_RB, m);
    ProfScope ps(p, FFB_KC_RING_FFT, s);
    // launched with programmatic serialization after the grid kernel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = dim3(32 * RFFT_RB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {ffb_pdl_attr()};
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int e = ffb_check_cuda(cudaLaunchKernelEx(&cfg, k_ring_fft<NTH, FMT>, Fpol, p->n_xi, p->k_max, o.lead,
                                                    (const float2 *)p->d_twT, (const float2 *)p->d_twA, o.p0, o.p1,
                                                    o.ld));
    p->launches++;
    return e;
}

template <int NTH>
static int launch_ring(ffb_plan_t p, int m, const float2 *Fpol, const RingOut &o, cudaStream_t s) {
    switch (o.fmt) {
        case FFB_FMT_F32: return launch_ring_fmt<NTH, FFB_FMT_F32>(p, m, Fpol, o, s);
        case FFB_FMT_TF32: return launch_ring_fmt<NTH, FFB_FMT_TF32>(p, m, Fpol, o, s);
        case FFB_FMT_TF32X2: return launch_ring_fmt<NTH, FFB_FMT_TF32X2>(p, m, Fpol, o, s);
        case FFB_FMT_BF16: return launch_ring_fmt<NTH, FFB_FMT_BF16>(p, m, Fpol, o, s);
        case FFB_FMT_BF16X2: return launch_ring_fmt<NTH, FFB_FMT_BF16X2>(p, m, Fpol, o, s);
        default: return FFB_ERR_ARG;
    }
}

int ffb_launch_ring_fft(ffb_plan_t p, int m, const float2 *Fpol, const RingOut &o, cudaStream_t s) {
    switch (p->n_theta) {
        case 128: return launch_ring<128>(p, m, Fpol, o, s);
        case 256: return launch_ring<256>(p, m, Fpol, o, s);
        case 512: return launch_ring<512>(p, m, Fpol, o, s);
        case 1024: return launch_ring<1024>(p, m, Fpol, o, s);
        default: return FFB_ERR_UNSUPPORTED;
    }
}
