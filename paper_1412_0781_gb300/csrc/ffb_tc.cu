// ffb_tc.cu -- step a5 (radial quadrature, Eq. a) on the tcgen05 tensor cores.
//
// For every k, D^(k) = A^(k) B^(k)T with A^(k) the (2 chunk) x n_xi ring
// spectra (rows = (image, re/im), contiguous per k) and B^(k) the p_k x n_xi
// radial table; both operands are K-major.  One CTA owns an M tile of 128 rows
// and one k:
//   * TMA (cp.async.bulk.tensor, 128-byte swizzle) brings all K of the A planes
//     and B planes into shared memory behind one mbarrier;
//   * one thread issues tcgen05.mma (M = 128, N = p_k rounded up to 16,
//     K = 8 (tf32) or 16 (bf16) per instruction) accumulating in TMEM, then
//     tcgen05.commit arrives on a second mbarrier;
//   * four warps read the 128 x N float32 accumulator with tcgen05.ld and write
//     the coefficients a_{k,q} (re/im rows) to the interleaved output.
//
// Precisions (hi/lo splitting, Markidis et al. 2018; Ootomo & Yokota 2022):
//   TF32    A (float32, truncated by the tensor core) x B_hi
//   TF32X3  A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = x rounded to tf32, lo = x - hi
//   BF16    A_hi B_hi with bf16 operands
//   BF16X3  A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = bf16(x), lo = bf16(x - hi)
// Every wait is bounded by a clock budget; a timeout latches FFB_ERR_TIMEOUT,
// waits (bounded) for in-flight copies, frees TMEM and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "ffb_internal.cuh"
#include "ffb_tc.cuh"

#define TC_BUDGET (4000000000LL)  // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;  // nearest, ties away
    return __uint_as_float(u);
}

// Bpad[plane][k][BN][n_xi]: rows q < p_k from B64, zero rows beyond.
template <bool BF16>
__global__ void k_prep_bpad(const double *__restrict__ B64, const int *__restrict__ pk_, const int *__restrict__ off_,
                            int kmax, int BN, int n_xi, void *hi, void *lo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(kmax + 1) * BN * n_xi;
    if (t >= tot) return;
    const int j = (int)(t % n_xi);
    const int q = (int)((t / n_xi) % BN);
    const int k = (int)(t / ((int64_t)n_xi * BN));
    double v = (q < pk_[k]) ? B64[(size_t)(off_[k] + q) * n_xi + j] : 0.0;
    if (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn((float)v);
        __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
        ((__nv_bfloat16 *)hi)[t] = h;
        ((__nv_bfloat16 *)lo)[t] = l;
    } else {
        float h = tf32_round((float)v);
        ((float *)hi)[t] = h;
        ((float *)lo)[t] = tf32_round((float)(v - (double)h));
    }
}

// ring spectra float32 -> operand planes (same [k][rows][n_xi] layout)
template <bool BF16, bool TWO>
__global__ void k_split_planes(const float *__restrict__ src, int64_t total, void *hi, void *lo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const float x = src[t];
    if (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        ((__nv_bfloat16 *)hi)[t] = h;
        if (TWO) ((__nv_bfloat16 *)lo)[t] = __float2bfloat16_rn(x - __bfloat162float(h));
    } else {
        const float h = tf32_round(x);
        ((float *)hi)[t] = h;
        if (TWO) ((float *)lo)[t] = x - h;
    }
}

// ---------------------------------------------------------------------------
// the contraction
// ---------------------------------------------------------------------------
template <int KIND, int NPA, int NPB, int NPROD>
__global__ void __launch_bounds__(128, 1)
k_tc_bessel(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
            const __grid_constant__ CUtensorMap mapB0, const __grid_constant__ CUtensorMap mapB1, int n_xi,
            int nimg, const int *__restrict__ pk_, const int *__restrict__ off_, int P, float *__restrict__ coef,
            int BNmax, int tmem_cols, int *status) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    constexpr int ES = (KIND == 0) ? 4 : 2;
    constexpr int KCH = 128 / ES;               // K elements per 128-byte row
    const int NCH = n_xi / KCH;
    const uint32_t a_bytes = 128u * 128u;       // one plane, one K chunk, 128 rows
    const uint32_t b_bytes = (uint32_t)BNmax * 128u;
    uint8_t *As = sm;
    uint8_t *Bs = sm + (size_t)NPA * NCH * a_bytes;
    uint64_t *bars = (uint64_t *)(Bs + (size_t)NPB * NCH * b_bytes);   // [0] loads, [1] mma done
    uint32_t *slot = (uint32_t *)(bars + 2);
    int *okflag = (int *)(slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x, k = blockIdx.y;
    const int pk = pk_[k], o = off_[k];
    const int BN = max(16, (pk + 15) & ~15);

    if (threadIdx.x == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
        *okflag = 1;
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, (uint32_t)tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;

    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(&bars[0], NPA * NCH * a_bytes + NPB * NCH * b_bytes);
        for (int ch = 0; ch < NCH; ++ch) {
            tc::tma_load_3d(As + (size_t)(0 * NCH + ch) * a_bytes, &mapA0, &bars[0], ch * KCH, 128 * m, k);
            if (NPA > 1) tc::tma_load_3d(As + (size_t)(1 * NCH + ch) * a_bytes, &mapA1, &bars[0], ch * KCH, 128 * m, k);
            tc::tma_load_3d(Bs + (size_t)(0 * NCH + ch) * b_bytes, &mapB0, &bars[0], ch * KCH, 0, k);
            if (NPB > 1) tc::tma_load_3d(Bs + (size_t)(1 * NCH + ch) * b_bytes, &mapB1, &bars[0], ch * KCH, 0, k);
        }
        if (!tc::mbar_wait(&bars[0], 0, TC_BUDGET)) {
            ffb_flag(status, FFB_ERR_TIMEOUT);
            *okflag = 0;
            tc::mbar_wait(&bars[0], 0, TC_BUDGET);  // let in-flight copies land
        } else {
            tc::fence_after_sync();
            const uint32_t id = tc::idesc(KIND == 0 ? 2 : 1, 128, BN);
            uint32_t acc = 0;
#pragma unroll
            for (int pr = 0; pr < NPROD; ++pr) {
                const int pa = (pr == 2) ? 1 : 0;   // products (0,0), (0,1), (1,0)
                const int pb = (pr == 1) ? 1 : 0;
                for (int ch = 0; ch < NCH; ++ch) {
                    const uint32_t a0 = tc::smem_u32(As + (size_t)(pa * NCH + ch) * a_bytes);
                    const uint32_t b0 = tc::smem_u32(Bs + (size_t)(pb * NCH + ch) * b_bytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = tc::desc_sw128(a0 + 32u * ks);
                        const uint64_t bd = tc::desc_sw128(b0 + 32u * ks);
                        if (KIND == 0) tc::mma_tf32(tbase, ad, bd, id, acc);
                        else tc::mma_bf16(tbase, ad, bd, id, acc);
                        acc = 1;
                    }
                }
            }
            tc::mma_commit(&bars[1]);
        }
    }
    __syncthreads();
    if (*okflag) {
        if (!tc::mbar_wait(&bars[1], 0, TC_BUDGET)) {
            ffb_flag(status, FFB_ERR_TIMEOUT);
            atomicExch(okflag, 0);
        }
    }
    tc::fence_after_sync();
    __syncthreads();
    if (*okflag) {
        const int r = 32 * warp + lane;            // accumulator row = TMEM lane
        const int R = 128 * m + r;
        const int img = R >> 1, cc = R & 1;
        for (int c16 = 0; c16 < BN; c16 += 16) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c16, v);
            if (img < nimg) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int q = c16 + i;
                    if (q < pk) coef[((size_t)img * P + o + q) * 2 + cc] = (k == 0 && cc == 1) ? 0.f : v[i];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, (uint32_t)tmem_cols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D map over [d2][d1][d0] elements, box (128 B of d0, box1 rows, 1)
static int make_map(CUtensorMap *map, void *base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t box1) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return FFB_ERR_CUDA;
    const uint64_t es = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {d0 * es, d0 * d1 * es};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), box1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r == CUDA_SUCCESS) ? FFB_OK : FFB_ERR_CUDA;
}

struct TcState {
    int prepared = -1;       // precision the tables were built for
    int BN = 0, tmem_cols = 0;
    void *bhi = nullptr, *blo = nullptr;   // padded radial tables
    void *ahi = nullptr, *alo = nullptr;   // split ring spectra
    CUtensorMap mA0, mA1, mB0, mB1;
};

static TcState *tc_state(ffb_plan_t p) {
    if (!p->tc) p->tc = new TcState();
    return (TcState *)p->tc;
}

void ffb_tc_release(ffb_plan_t p) {
    if (!p->tc) return;
    TcState *t = (TcState *)p->tc;
    void *ptrs[] = {t->bhi, t->blo, t->ahi, t->alo};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete t;
    p->tc = nullptr;
}

static int tc_prepare(ffb_plan_t p, cudaStream_t s) {
    TcState *t = tc_state(p);
    if (t->prepared == p->precision) return FFB_OK;
    const bool bf16 = (p->precision == FFB_BF16 || p->precision == FFB_BF16X3);
    const size_t es = bf16 ? 2 : 4;
    const int kch = (int)(128 / es);
    if (p->n_xi % kch) return FFB_ERR_UNSUPPORTED;
    t->BN = (p->pmax + 15) & ~15;
    if (t->BN > 256) return FFB_ERR_UNSUPPORTED;
    t->tmem_cols = 32;
    while (t->tmem_cols < t->BN) t->tmem_cols <<= 1;
    for (void **q : {&t->bhi, &t->blo, &t->ahi, &t->alo})
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    const size_t nb = (size_t)(p->k_max + 1) * t->BN * p->n_xi;
    const size_t na = (size_t)(p->k_max + 1) * p->chunk * 2 * p->n_xi;
    int e;
    if ((e = ffb_check_cuda(cudaMalloc(&t->bhi, nb * es)))) return e;
    if ((e = ffb_check_cuda(cudaMalloc(&t->blo, nb * es)))) return e;
    if ((e = ffb_check_cuda(cudaMalloc(&t->ahi, na * es)))) return e;
    if ((e = ffb_check_cuda(cudaMalloc(&t->alo, na * es)))) return e;
    const unsigned g = (unsigned)((nb + 255) / 256);
    if (bf16) k_prep_bpad<true><<<g, 256, 0, s>>>(p->d_B64, p->d_p, p->d_off, p->k_max, t->BN, p->n_xi, t->bhi, t->blo);
    else k_prep_bpad<false><<<g, 256, 0, s>>>(p->d_B64, p->d_p, p->d_off, p->k_max, t->BN, p->n_xi, t->bhi, t->blo);
    p->launches++;
    if ((e = ffb_check_cuda(cudaGetLastError()))) return e;
    const uint64_t rows = 2ull * p->chunk;
    // plain TF32 reads the float32 spectra directly
    void *a0 = (p->precision == FFB_TF32) ? (void *)p->d_Fhat : t->ahi;
    if ((e = make_map(&t->mA0, a0, bf16, p->n_xi, rows, p->k_max + 1, 128))) return e;
    if ((e = make_map(&t->mA1, t->alo, bf16, p->n_xi, rows, p->k_max + 1, 128))) return e;
    if ((e = make_map(&t->mB0, t->bhi, bf16, p->n_xi, t->BN, p->k_max + 1, t->BN))) return e;
    if ((e = make_map(&t->mB1, t->blo, bf16, p->n_xi, t->BN, p->k_max + 1, t->BN))) return e;
    t->prepared = p->precision;
    return FFB_OK;
}

template <int KIND, int NPA, int NPB, int NPROD>
static int launch_tc(ffb_plan_t p, TcState *t, int nimg, float *d_coef_chunk, cudaStream_t s) {
    const int es = (KIND == 0) ? 4 : 2;
    const int nch = p->n_xi / (128 / es);
    const size_t smem = 1024 + (size_t)NPA * nch * 128 * 128 + (size_t)NPB * nch * t->BN * 128 + 64;
    static int attr = 0;
    if (attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_tc_bessel<KIND, NPA, NPB, NPROD>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    dim3 g((2 * nimg + 127) / 128, p->k_max + 1);
    ProfScope ps(p, FFB_KC_BESSEL, s);
    k_tc_bessel<KIND, NPA, NPB, NPROD><<<g, 128, smem, s>>>(t->mA0, t->mA1, t->mB0, t->mB1, p->n_xi, nimg, p->d_p,
                                                           p->d_off, p->P, d_coef_chunk, t->BN, t->tmem_cols,
                                                           p->d_status);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// shared memory of one CTA: all K of the A and B planes must fit
bool ffb_tc_supported(ffb_plan_t p) {
    const bool bf16 = (p->precision == FFB_BF16 || p->precision == FFB_BF16X3);
    const bool two = (p->precision == FFB_BF16X3 || p->precision == FFB_TF32X3);
    const int es = bf16 ? 2 : 4;
    if (p->n_xi % (128 / es)) return false;
    const int nch = p->n_xi / (128 / es);
    const int BN = (p->pmax + 15) & ~15;
    if (BN > 256) return false;
    const size_t smem = 1024 + (size_t)(two ? 2 : 1) * nch * 128 * 128 + (size_t)(two ? 2 : 1) * nch * BN * 128 + 64;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return smem <= (size_t)optin;
}

int ffb_launch_bessel_tc(ffb_plan_t p, int nimg, float *d_coef_chunk, cudaStream_t s) {
    int e = tc_prepare(p, s);
    if (e) return e;
    TcState *t = tc_state(p);
    const int64_t total = (int64_t)(p->k_max + 1) * p->chunk * 2 * p->n_xi;
    const unsigned g = (unsigned)((total + 255) / 256);
    if (p->precision != FFB_TF32) {
        ProfScope ps(p, FFB_KC_BESSEL, s);
        switch (p->precision) {
            case FFB_TF32X3: k_split_planes<false, true><<<g, 256, 0, s>>>(p->d_Fhat, total, t->ahi, t->alo); break;
            case FFB_BF16: k_split_planes<true, false><<<g, 256, 0, s>>>(p->d_Fhat, total, t->ahi, t->alo); break;
            default: k_split_planes<true, true><<<g, 256, 0, s>>>(p->d_Fhat, total, t->ahi, t->alo); break;
        }
        p->launches++;
        if ((e = ffb_check_cuda(cudaGetLastError()))) return e;
    }
    switch (p->precision) {
        case FFB_TF32: return launch_tc<0, 1, 1, 1>(p, t, nimg, d_coef_chunk, s);
        case FFB_TF32X3: return launch_tc<0, 2, 2, 3>(p, t, nimg, d_coef_chunk, s);
        case FFB_BF16: return launch_tc<1, 1, 1, 1>(p, t, nimg, d_coef_chunk, s);
        case FFB_BF16X3: return launch_tc<1, 2, 2, 3>(p, t, nimg, d_coef_chunk, s);
        default: return FFB_ERR_ARG;
    }
}
