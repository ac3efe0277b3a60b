// ffb_gemm.cu -- the dense contractions of the hot path on CUDA cores (FP32):
//   a5  radial quadrature (Eq. a):  a^(k)_{i,q} = sum_j Fhat^(k)_{i,j} B^(k)_{q,j}
//   a6  k = 0 mean (Alg. 2 step 1, Eq. mean2)
//   a7  covariance blocks (Eqs. ck, ck_0): sum_i Re(a_{i,q} conj a_{i,q'})
// plus the finalisation C^(k) = acc/n (k = 0 centred).
#include "ffb_internal.cuh"

// ---------------------------------------------------------------------------
// a5, FP32: one CTA per (k, 32 images).  Rows of the A operand are the 64
// (image, re/im) rows of Fhat[k] (contiguous in memory), columns of B are
// the p_k rows of B^(k) in tiles of 64; K = n_xi, in slabs of at most
// BES_KT (one slab up to L = 384 at R = L/2).  Both tiles are stored
// transposed in shared memory (K-major: At[j][row], Bt[j][q]) so that a
// thread reads its 4 rows and 4 columns with two 16-byte loads per j.
// Thread (ty = t % 16, tx = t / 16): rows 4 ty .., columns 4 tx ..; a warp
// spans 8 columns, so warps whose columns lie past p_k skip the products.
// ---------------------------------------------------------------------------
#define BES_IMG 32
#define BES_TP 68    // row pitch of the transposed tiles (floats): 64 + 4, 16-byte aligned
#define BES_KT 384   // K slab: two [BES_KT][BES_TP] float tiles = 204 KB

static int bessel_fp32_kt(int n_xi) { return n_xi < BES_KT ? n_xi : BES_KT; }
static size_t bessel_fp32_smem(int n_xi) { return sizeof(float) * (size_t)bessel_fp32_kt(n_xi) * 2 * BES_TP; }

__global__ void __launch_bounds__(256)
k_bessel_fp32(const float *__restrict__ Fhat, const float *__restrict__ Bf, const int *__restrict__ pk_,
              const int *__restrict__ off_, int n_xi, int kt, int chunk, int nimg, int P,
              float2 *__restrict__ coef) {
    extern __shared__ float4 sm4[];
    float *At = (float *)sm4;                    // [kt][BES_TP]
    float *Bt = At + (size_t)kt * BES_TP;        // [kt][BES_TP]
    const int k = blockIdx.y;
    const int pk = pk_[k], o = off_[k];
    const int i0 = blockIdx.x * BES_IMG;
    const float *Ak = Fhat + ((size_t)k * chunk + i0) * 2 * n_xi;
    const int rows = min(BES_IMG, nimg - i0) * 2;
    const bool one_slab = kt >= n_xi;
    auto load_a = [&](int j0, int kl) {
        for (int e = threadIdx.x; e < 2 * BES_IMG * kl; e += 256) {
            const int r = e / kl, j = e - r * kl;
            At[j * BES_TP + r] = (r < rows) ? __ldg(&Ak[(size_t)r * n_xi + j0 + j]) : 0.f;
        }
    };
    if (one_slab) load_a(0, n_xi);
    const int ty = threadIdx.x & 15, tx = threadIdx.x >> 4;
    for (int q0 = 0; q0 < pk; q0 += 64) {
        const bool active = 8 * (threadIdx.x >> 5) < pk - q0;   // else the warp's 8 columns are padding
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        for (int j0 = 0; j0 < n_xi; j0 += kt) {
            const int kl = min(kt, n_xi - j0);
            __syncthreads();
            if (!one_slab) load_a(j0, kl);
            for (int e = threadIdx.x; e < 64 * kl; e += 256) {
                const int q = e / kl, j = e - q * kl;
                Bt[j * BES_TP + q] = (q0 + q < pk) ? __ldg(&Bf[(size_t)(o + q0 + q) * n_xi + j0 + j]) : 0.f;
            }
            __syncthreads();
            if (!active) continue;
#pragma unroll 4
            for (int j = 0; j < kl; ++j) {
                const float4 a = *(const float4 *)&At[j * BES_TP + 4 * ty];
                const float4 b = *(const float4 *)&Bt[j * BES_TP + 4 * tx];
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
            }
        }
        if (!active) continue;
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {             // rows 4 ty + 2 ii (re), + 1 (im)
            const int img = i0 + 2 * ty + ii;
            if (img >= nimg) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int q = q0 + 4 * tx + c;
                if (q < pk) coef[(size_t)img * P + o + q] = make_float2(acc[2 * ii][c], (k == 0) ? 0.f : acc[2 * ii + 1][c]);
            }
        }
    }
}

int ffb_launch_bessel_fp32(ffb_plan_t p, int nimg, float *d_coef_chunk, cudaStream_t s) {
    const size_t smem = bessel_fp32_smem(p->n_xi);
    static int attr = 0;
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_bessel_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((nimg + BES_IMG - 1) / BES_IMG, p->k_max + 1);
    ProfScope ps(p, FFB_KC_BESSEL, s);
    k_bessel_fp32<<<g, 256, smem, s>>>(p->d_Fhat, p->d_Bf, p->d_p, p->d_off, p->n_xi, bessel_fp32_kt(p->n_xi),
                                       p->chunk, nimg, p->P, (float2 *)d_coef_chunk);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

int ffb_launch_bessel(ffb_plan_t p, int nimg, float *d_coef_chunk, bool planes_ready, cudaStream_t s) {
    if (p->precision != FFB_FP32) return ffb_launch_bessel_tc(p, nimg, d_coef_chunk, planes_ready, s);
    return ffb_launch_bessel_fp32(p, nimg, d_coef_chunk, s);
}

// ---------------------------------------------------------------------------
// a6/a7: covariance accumulation in float32 tiles.  A persistent CTA walks the
// items of a stack table (CovGroup): item = (stack, tile (k, q0, q1) of the
// stack's tile list, image range).  The tile is the 64 x 64 block of C^(k) at
// rows q0.., columns q1..; each thread owns a 4 x 4 sub-tile, sums 128 images
// in float32 and folds the partial sums into float64 registers; the result is
// added to the float64 accumulator with atomics (both the tile and, off the
// diagonal, its transpose).  For k = 0 the values are shifted by `shift` (a
// pilot mean): sum (a - s)(a - s)^T, finalised as C = acc/n - d d^T with
// d = sum(a - s)/n; the diagonal tiles of block 0 also accumulate sum(a - s).
// ---------------------------------------------------------------------------
#define COV_TI 32
__global__ void __launch_bounds__(256)
k_cov_fp32(const __grid_constant__ CovGroup g) {
    __shared__ float2 Xa[COV_TI][64];
    __shared__ float2 Xb[COV_TI][64];
    // warp w owns rows 16 (w % 4) .. + 15 and columns 32 (w / 4) .. + 31 of the
    // 64 x 64 tile, 4 x 4 per thread; a warp whose sub-block lies past p_k skips
    // the products (uniformly), so small blocks cost less than a full tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0w = 16 * (warp & 3) + 4 * (lane >> 3);
    const int c0w = 32 * (warp >> 2) + 4 * (lane & 7);
    for (int64_t item = blockIdx.x; item < g.nitems; item += gridDim.x) {
        const CovStack &S = g.st[cov_stack_of(g, item)];
        const int64_t local = item - S.item0;
        const int4 wk = S.work[local % S.nk];
        const int k = wk.x, q0 = wk.y, q1 = wk.z;
        const int pk = S.pk[k], o = S.off[k];
        const int64_t ib = (local / S.nk) * (int64_t)S.per;
        const int64_t ie = min(S.n, ib + (int64_t)S.per);
        const float2 *coef = S.coef;
        const int P = S.P;
        const float *shift = S.shift;
        const bool do_sum = (k == 0 && q0 == q1);  // diagonal tiles of block 0 carry the mean
        const bool diag = (q0 == q1);              // X_b = X_a: staged once
        float accf[4][4], hi[4][4], lo[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) accf[r][c] = hi[r][c] = lo[r][c] = 0.f;
        float sf = 0.f;
        double sd = 0.0;
        int tiles = 0;
        // the next tile's values are fetched into registers while this tile's
        // products run: thread t stages entries e = t + 256 u of the 32 x 64
        // block (image e / 64, column e % 64)
        float2 pa[COV_TI * 64 / 256], pb[COV_TI * 64 / 256];
        auto fetch = [&](int64_t i) {
#pragma unroll
            for (int u = 0; u < COV_TI * 64 / 256; ++u) {
                const int e = threadIdx.x + 256 * u, ii = e >> 6, qq = e & 63;
                const int64_t img = i + ii;
                float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
                if (img < ie) {
                    if (q0 + qq < pk) va = __ldg(&coef[img * P + o + q0 + qq]);
                    if (!diag && q1 + qq < pk) vb = __ldg(&coef[img * P + o + q1 + qq]);
                }
                pa[u] = va;
                pb[u] = vb;
            }
        };
        if (ib < ie) fetch(ib);
        for (int64_t i = ib; i < ie; i += COV_TI) {
            __syncthreads();
#pragma unroll
            for (int u = 0; u < COV_TI * 64 / 256; ++u) {
                const int e = threadIdx.x + 256 * u, ii = e >> 6, qq = e & 63;
                float2 va = pa[u], vb = pb[u];
                if (k == 0 && i + ii < ie) {
                    va = make_float2(q0 + qq < pk ? va.x - shift[q0 + qq] : 0.f, 0.f);
                    vb = make_float2(q1 + qq < pk && !diag ? vb.x - shift[q1 + qq] : 0.f, 0.f);
                }
                Xa[ii][qq] = va;
                if (!diag) Xb[ii][qq] = vb;
            }
            __syncthreads();
            if (i + COV_TI < ie) fetch(i + COV_TI);
            const float2(*Xs)[64] = diag ? Xa : Xb;
            if (16 * (warp & 3) < pk - q0 && 32 * (warp >> 2) < pk - q1) {
#pragma unroll 4
                for (int ii = 0; ii < COV_TI; ++ii) {
                    float2 a[4], bq[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = Xa[ii][r0w + r];
#pragma unroll
                    for (int c = 0; c < 4; ++c) bq[c] = Xs[ii][c0w + c];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            accf[r][c] = fmaf(a[r].x, bq[c].x, fmaf(a[r].y, bq[c].y, accf[r][c]));
                }
            }
            if (do_sum && threadIdx.x < 64) {
                for (int ii = 0; ii < COV_TI; ++ii) sf += Xa[ii][threadIdx.x].x;
            }
            if (++tiles == 4) {
                // fold the 128-image partials into a compensated float32 sum
                // (TwoSum; float64 arithmetic runs at a small fraction of the
                // float32 rate on this GPU)
                tiles = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float x = accf[r][c], s2 = hi[r][c] + x, bp = s2 - hi[r][c];
                        lo[r][c] += (hi[r][c] - (s2 - bp)) + (x - bp);
                        hi[r][c] = s2;
                        accf[r][c] = 0.f;
                    }
                sd += (double)sf;
                sf = 0.f;
            }
        }
        double *blk = S.acc + S.cov_off[k];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int qa = q0 + r0w + r, qb = q1 + c0w + c;
                if (qa < pk && qb < pk) {
                    const double v = (double)hi[r][c] + (double)lo[r][c] + (double)accf[r][c];
                    atomicAdd(&blk[(size_t)qa * pk + qb], v);
                    if (q0 != q1) atomicAdd(&blk[(size_t)qb * pk + qa], v);
                }
            }
        if (do_sum && threadIdx.x < 64 && q0 + (int)threadIdx.x < pk)
            atomicAdd(&S.sum0[q0 + threadIdx.x], sd + (double)sf);
    }
}

void ffb_cov_stack(ffb_plan_t p, const float *d_coef, int64_t n, bool tc, CovStack *st) {
    st->coef = (const float2 *)d_coef;
    st->n = n;
    st->item0 = 0;
    st->pk = p->d_p;
    st->off = p->d_off;
    st->cov_off = p->d_cov_off;
    st->work = tc ? p->d_cov_sb : p->d_cov_work;
    st->shift = p->d_shift;
    st->acc = p->d_acc;
    st->sum0 = p->d_sum0;
    st->P = p->P;
    st->nk = tc ? p->n_cov_sb : p->n_cov_work;
    st->per = tc ? 512 : 2048;
    st->pmax = p->pmax;
}

int ffb_cov_grid_default(int precision) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (precision != FFB_FP32) return sms;   // one CTA per SM: it holds all 512 TMEM columns
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cov_fp32, 256, 0);
    return sms * (occ > 0 ? occ : 1);
}

int ffb_launch_cov_group(int precision, const CovGroup &g, int grid, int *status, cudaStream_t s) {
    if (g.S < 1 || g.S > FFB_GROUP_MAX) return FFB_ERR_ARG;
    if (g.nitems <= 0) return FFB_OK;
    if (precision != FFB_FP32) return ffb_launch_cov_group_tc(precision, g, grid, status, s);
    if (grid <= 0) grid = ffb_cov_grid_default(precision);
    if ((int64_t)grid > g.nitems) grid = (int)g.nitems;
    k_cov_fp32<<<grid, 256, 0, s>>>(g);
    return ffb_check_cuda(cudaGetLastError());
}

// pilot shift for the k = 0 block: mean of Re a_{i,0,q} over the first
// min(n, 512) images of the first batch after a reset (any shift near the
// mean keeps the shifted sums well conditioned; C = acc/n - d d^T is exact for
// every shift).  Block of 4 x 64 threads: q = threadIdx.x % 64 within the
// block's 64 rows, image group threadIdx.x / 64 (every fourth image).
__global__ void __launch_bounds__(256) k_cov_shift(const float2 *__restrict__ coef, int64_t n, int P, int p0,
                                                   float *shift) {
    __shared__ float part[4][64];
    const int qq = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int q = blockIdx.x * 64 + qq;
    const int m = (int)min(n, (int64_t)512);
    float s0 = 0.f, s1 = 0.f;
    if (q < p0) {
        int i = grp;
        for (; i + 4 < m; i += 8) {
            s0 += coef[(int64_t)i * P + q].x;
            s1 += coef[(int64_t)(i + 4) * P + q].x;
        }
        if (i < m) s0 += coef[(int64_t)i * P + q].x;
    }
    part[grp][qq] = s0 + s1;
    __syncthreads();
    if (grp == 0 && q < p0) shift[q] = (part[0][qq] + part[1][qq] + part[2][qq] + part[3][qq]) / (float)m;
}

// C^(k) = acc^(k)/n; for k = 0: C = acc/n - d d^T, mean = shift + d, d = sum0/n
__global__ void k_cov_final(const double *__restrict__ acc, const double *__restrict__ sum0,
                            const float *__restrict__ shift, double n, const int *__restrict__ pk_,
                            const int *__restrict__ cov_off, double *__restrict__ Cfin, double *__restrict__ mean) {
    const int k = blockIdx.y;
    const int pk = pk_[k];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= pk * pk) return;
    const int qa = e / pk, qb = e % pk;
    // symmetric part: tensor-core partial sums of (a, b) and (b, a) round differently
    double v = 0.5 * (acc[cov_off[k] + e] + acc[cov_off[k] + qb * pk + qa]) / n;
    if (k == 0) {
        double da = sum0[qa] / n, db = sum0[qb] / n;
        v -= da * db;
        if (qb == 0) mean[qa] = (double)shift[qa] + da;
    }
    Cfin[cov_off[k] + e] = v;
}

int ffb_launch_cov_shift(ffb_plan_t p, const float *d_coef, int64_t n, cudaStream_t s) {
    ProfScope ps(p, FFB_KC_COVAUX, s);
    k_cov_shift<<<(p->p[0] + 63) / 64, 256, 0, s>>>((const float2 *)d_coef, n, p->P, p->p[0], p->d_shift);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

int ffb_launch_cov(ffb_plan_t p, const float *d_coef, int64_t n, cudaStream_t s) {
    if (ffb_tc_cov_supported(p)) return ffb_launch_cov_tc(p, d_coef, n, s);
    CovGroup g;          // copied into the launch's parameters
    g.S = 1;
    g.tile_imgs = 32;
    ffb_cov_stack(p, d_coef, n, false, &g.st[0]);
    g.nitems = (int64_t)g.st[0].nk * ((n + g.st[0].per - 1) / g.st[0].per);
    ProfScope ps(p, FFB_KC_COV, s);
    const int e = ffb_launch_cov_group(FFB_FP32, g, 0, p->d_status, s);
    p->launches++;
    return e;
}

int ffb_launch_cov_final(ffb_plan_t p, cudaStream_t s) {
    if (p->n_acc <= 0) return FFB_ERR_STATE;
    dim3 g((p->pmax * p->pmax + 255) / 256, p->k_max + 1);
    ProfScope ps(p, FFB_KC_COVAUX, s);
    k_cov_final<<<g, 256, 0, s>>>(p->d_acc, p->d_sum0, p->d_shift, (double)p->n_acc, p->d_p, p->d_cov_off,
                                  p->d_Cfin, p->d_mean);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// a9: steerable filter.  M^(k) = U^(k) diag(h^(k)) U^(k)T (one CTA per k), then
// a_out = W_k (M^(k) (a - m) + m) with m the k = 0 mean (zero for k > 0) and
// W_k = 1 (k = 0), 2 (k > 0), i.e. the coefficients of the filtered image
// ready for the synthesis S = T W (Eq. sPCAcoeff filtered and recombined).
// ---------------------------------------------------------------------------
__global__ void k_filter_matrix(const double *__restrict__ U, const double *__restrict__ gain,
                                const int *__restrict__ pk_, const int *__restrict__ off_,
                                const int *__restrict__ cov_off, float *__restrict__ M) {
    const int k = blockIdx.x;
    const int pk = pk_[k], o = off_[k];
    const double *Uk = U + cov_off[k];
    for (int e = threadIdx.x; e < pk * pk; e += blockDim.x) {
        const int a = e / pk, b = e % pk;
        double s = 0.0;
        for (int l = 0; l < pk; ++l) s += Uk[a * pk + l] * gain[o + l] * Uk[b * pk + l];
        M[cov_off[k] + e] = (float)s;
    }
}

#define FIL_IMG 32
__global__ void __launch_bounds__(256)
k_filter(const float2 *__restrict__ cin, float2 *__restrict__ cout, int64_t n, int P, const float *__restrict__ M,
         const double *__restrict__ mean, const int *__restrict__ pk_, const int *__restrict__ off_,
         const int *__restrict__ cov_off, int flags, int mglobal) {
    extern __shared__ float smf[];
    const int k = blockIdx.y;
    const int pk = pk_[k], o = off_[k];
    const int64_t i0 = (int64_t)blockIdx.x * FIL_IMG;
    const bool affine = !(flags & 1) && k == 0;
    // float2 tile first: it needs 8-byte alignment (pk * pk floats may be odd);
    // M^(k) is staged behind it unless it is read from global memory (blocks
    // whose pk x pk floats do not fit next to the tile)
    float2 *X = (float2 *)smf;                    // [FIL_IMG][pk]
    const float *Ms = M + cov_off[k];             // [pk][pk]
    if (!mglobal) {
        float *Mst = smf + 2 * FIL_IMG * pk;
        for (int e = threadIdx.x; e < pk * pk; e += blockDim.x) Mst[e] = Ms[e];
        Ms = Mst;
    }
    for (int t = threadIdx.x; t < FIL_IMG * pk; t += blockDim.x) {
        const int ii = t / pk, q = t - ii * pk;
        float2 v = make_float2(0.f, 0.f);
        if (i0 + ii < n) {
            v = cin[(i0 + ii) * P + o + q];
            if (k == 0) v.y = 0.f;
            if (affine) v.x -= (float)mean[q];
        }
        X[t] = v;
    }
    __syncthreads();
    const float wk = ((flags & 2) && k > 0) ? 2.f : 1.f;
    for (int t = threadIdx.x; t < FIL_IMG * pk; t += blockDim.x) {
        const int ii = t / pk, a = t - ii * pk;
        if (i0 + ii >= n) continue;
        float sx = 0.f, sy = 0.f;
        for (int b = 0; b < pk; ++b) {
            const float m = Ms[a * pk + b];
            const float2 x = X[ii * pk + b];
            sx = fmaf(m, x.x, sx);
            sy = fmaf(m, x.y, sy);
        }
        if (affine) sx += (float)mean[a];
        cout[(i0 + ii) * P + o + a] = make_float2(wk * sx, wk * sy);
    }
}

__global__ void k_weight(const float2 *__restrict__ cin, float2 *__restrict__ cout, int64_t total, int P, int p0) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int q = (int)(t % P);
    float2 v = cin[t];
    if (q < p0) v.y = 0.f;
    const float wk = (q < p0) ? 1.f : 2.f;
    cout[t] = make_float2(wk * v.x, wk * v.y);
}

int ffb_launch_filter_matrix(ffb_plan_t p, cudaStream_t s) {
    ProfScope ps(p, FFB_KC_FILTER, s);
    k_filter_matrix<<<p->k_max + 1, 256, 0, s>>>(p->d_evecs, p->d_gain, p->d_p, p->d_off, p->d_cov_off, p->d_M);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

int ffb_launch_filter(ffb_plan_t p, const float *d_coef_in, int64_t n, float *d_coef_out, int flags,
                      cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t tile = sizeof(float2) * FIL_IMG * (size_t)p->pmax;
    const size_t mbytes = sizeof(float) * (size_t)p->pmax * p->pmax;
    const int mglobal = (tile + mbytes > (size_t)optin) ? 1 : 0;
    const size_t smem = mglobal ? tile : tile + mbytes;
    static int attr = 0;
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((unsigned)((n + FIL_IMG - 1) / FIL_IMG), p->k_max + 1);
    ProfScope ps(p, FFB_KC_FILTER, s);
    k_filter<<<g, 256, smem, s>>>((const float2 *)d_coef_in, (float2 *)d_coef_out, n, p->P, p->d_M, p->d_mean,
                                  p->d_p, p->d_off, p->d_cov_off, flags, mglobal);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

int ffb_launch_weight(ffb_plan_t p, const float *d_coef_in, int64_t n, float *d_coef_out, cudaStream_t s) {
    const int64_t total = n * (int64_t)p->P;
    ProfScope ps(p, FFB_KC_FILTER, s);
    k_weight<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const float2 *)d_coef_in, (float2 *)d_coef_out, total,
                                                           p->P, p->p[0]);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}
