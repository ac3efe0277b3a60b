// ffb_tc.cu -- steps a5 (radial quadrature, Eq. a) and a6/a7 (covariance,
// Eqs. ck, ck_0) on the tcgen05 tensor cores.
//
// Quadrature: for every k, D^(k) = A^(k) B^(k)T with A^(k) the ring spectra of
// a group of chunks (rows = (image, re/im), contiguous per k; the ring FFT
// writes them as operand planes) and B^(k) the p_k x n_xi radial table; both
// operands K-major.  A persistent, warp-specialised CTA walks the (k, M tile
// of 128 rows) items:
//   * warp 0 streams the 128-byte K chunks of A and B (hi/lo planes) by TMA
//     (cp.async.bulk.tensor, 128-byte swizzle) through a ring of stages with
//     full/empty mbarriers;
//   * warp 1 allocates TMEM and one thread issues tcgen05.mma (M = 128,
//     N = p_k rounded up to 16, K = 8 (tf32) or 16 (bf16) per instruction)
//     into one of two alternating accumulators;
//   * eight epilogue warps read an accumulator with tcgen05.ld, release it and
//     write the coefficients a_{k,q} (re/im rows) to the interleaved output.
// Covariance: see the section below (super-blocks of consecutive k).
//
// Precisions (hi/lo splitting, Markidis et al. 2018; Ootomo & Yokota 2022):
//   TF32    A (float32, truncated by the tensor core) x B_hi
//   TF32X3  A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = x rounded to tf32, lo = x - hi
//   BF16    A_hi B_hi with bf16 operands
//   BF16X3  A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = bf16(x), lo = bf16(x - hi)
// Every wait is bounded by a clock budget; a timeout latches FFB_ERR_TIMEOUT,
// waits (bounded, with the full default budget) for the copies and MMAs it
// has issued, frees TMEM and returns.  The waits between the pipeline roles
// take the plan's budget `wb` (the default unless a test shortens it).
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "ffb_internal.cuh"
#include "ffb_tc.cuh"

// operand planes of one quadrature group: 4 BF16x3 chunks at L = 128 (114 MB;
// measured 1.7 % faster per step than 2 chunks in 64 MiB, though the planes
// and the polar buffer then exceed L2; with the L2 eviction hints of the
// pixel, polar-buffer and plane accesses, 4 chunks 1,194 k images/s, 2 chunks
// 1,175 k, 1 chunk 1,169 k)
#ifndef FFB_PLANE_BUDGET_MB
#define FFB_PLANE_BUDGET_MB 128
#endif

#define TC_BUDGET FFB_WAIT_BUDGET   // drains of issued copies and MMAs

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
// Bpad[plane][k][BN][ld]: rows q < p_k, columns j < n_xi from B64, zero
// elsewhere (ld = n_xi rounded up to whole 128-byte K chunks).
template <bool BF16>
__global__ void k_prep_bpad(const double *__restrict__ B64, const int *__restrict__ pk_, const int *__restrict__ off_,
                            int kmax, int BN, int n_xi, int ld, void *hi, void *lo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(kmax + 1) * BN * ld;
    if (t >= tot) return;
    const int j = (int)(t % ld);
    const int q = (int)((t / ld) % BN);
    const int k = (int)(t / ((int64_t)ld * BN));
    double v = (q < pk_[k] && j < n_xi) ? B64[(size_t)(off_[k] + q) * n_xi + j] : 0.0;
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

// ring spectra float32 [k][rows][n_xi] -> operand planes [k][rows][ld]
// (separate-kernel path; the fused path's ring FFT writes the planes itself)
template <bool BF16, bool TWO>
__global__ void k_split_planes(const float *__restrict__ src, int64_t total, int n_xi, int ld, void *hi, void *lo) {
    const int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s0 >= total) return;
    const float x = src[s0];
    const int64_t t = (s0 / n_xi) * ld + (s0 % n_xi);
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
#define TCB_EPI 8     // epilogue warps: two per TMEM lane quarter
#define TCB_WARPS (2 + TCB_EPI)   // warp 0: TMA, warp 1: MMA and TMEM, the rest: epilogue

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(32 * TCB_EPI) : "memory"); }

// One stack of a quadrature launch: the TMA maps of its ring-spectrum planes
// (A, hi and lo) and of its padded radial table (B, hi and lo), and where its
// items' coefficients go.  A single plan's launch passes one as a kernel
// parameter; a group's launch reads an array of them from device memory
// (written once per group call shape), stack s owning items
// item0 .. item0 + (k_max + 1) nM - 1.
struct TcStack {
    CUtensorMap mA0, mA1, mB0, mB1;
    const int *pk, *off;   // p_k and coefficient offsets of the stack's plan (device)
    float *coef;           // coefficients of the launch's first image of the stack
    int P, nimg, nM, NCH;  // coefficients per image, images, M tiles, 128-byte K chunks
    int item0;
    int BN;                // rows of the B map's box (<= the launch's BNmax)
    int pad_[2];
};

// the stack of `item`: the launch's one stack, or, in a group, the last stack
// whose first item is <= item (a CTA's items rise, so the search only moves on)
template <bool GROUP>
__device__ __forceinline__ const TcStack *tc_stack_of(const TcStack &one, const TcStack *__restrict__ many, int S,
                                                      int item, int &s) {
    if constexpr (!GROUP) {
        return &one;
    } else {
        while (s + 1 < S && item >= __ldg(&many[s + 1].item0)) ++s;
        return &many[s];
    }
}

// Persistent: CTA b takes items b, b + gridDim.x, ... of the (stack, k, M
// tile) list (item = item0 + k nM + m; M tile m = images 64 m .. 64 m + 63,
// rows image x re/im).  For every item the producer streams the K chunks of
// A and B (hi/lo planes) through a ring of nst stages (full/empty
// mbarriers); the MMA thread accumulates each item into one of two TMEM
// accumulators and commits it to the epilogue (accf), which drains it with
// tcgen05.ld into a padded [64 images][BN q][re, im] stage, releases the
// accumulator (acce) and writes the coefficients as contiguous runs per
// image.  BNmax and acc_cols cover the widest stack of the launch.
template <int KIND, int NPA, int NPB, int NPROD, bool GROUP>
__global__ void __launch_bounds__(32 * TCB_WARPS)
k_tc_bessel(const __grid_constant__ TcStack one, const TcStack *__restrict__ many, int S, int BNmax, int acc_cols,
            int nst, int nitems, int *status, long long wb) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    constexpr int ES = (KIND == 0) ? 4 : 2;
    constexpr int KCH = 128 / ES;               // K elements per 128-byte row
    const uint32_t a_bytes = 128u * 128u;       // one plane, one K chunk, 128 rows
    const uint32_t b_bytes = (uint32_t)BNmax * 128u;
    const uint32_t st_bytes = NPA * a_bytes + NPB * b_bytes;   // one stage: every plane of one K chunk
    const int ldst = 2 * BNmax + 2;             // floats per image row of the epilogue stage
    float *stage = (float *)(sm + (size_t)nst * st_bytes);
    const size_t stage_bytes = ((size_t)64 * ldst * 4 + 15) & ~(size_t)15;
    uint64_t *bars = (uint64_t *)(sm + (size_t)nst * st_bytes + stage_bytes);
    uint64_t *full = bars, *empty = bars + nst, *accf = bars + 2 * nst, *acce = bars + 2 * nst + 2;
    uint32_t *slot = (uint32_t *)(bars + 2 * nst + 4);
    int *okflag = (int *)(slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int myitems = (blockIdx.x < nitems) ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    pdl_trigger();

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * nst; ++i) tc::mbar_init(&bars[i], 1);
        tc::mbar_init(&accf[0], 1);
        tc::mbar_init(&accf[1], 1);
        tc::mbar_init(&acce[0], TCB_EPI);   // one arrival per epilogue warp
        tc::mbar_init(&acce[1], TCB_EPI);
        tc::fence_mbar_init();
        *okflag = 1;
    }
    if (warp == 1) {
        tc::tmem_alloc(slot, (uint32_t)(2 * acc_cols));
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;

    if (warp == 0) {
        if (lane == 0) {                                  // ---- TMA producer
            pdl_wait();   // the operand planes come from the previous kernels
            int64_t g = 0;
            bool ok = true;
            int si = 0, seen = -1;
            for (int it = 0; it < myitems && ok && *(volatile int *)okflag; ++it) {
                const int item = blockIdx.x + it * gridDim.x;
                const TcStack *st = tc_stack_of<GROUP>(one, many, S, item, si);
                if (GROUP && si != seen) {   // maps written to device memory before the launch
                    tc::tmap_acquire(&st->mA0);
                    tc::tmap_acquire(&st->mA1);
                    tc::tmap_acquire(&st->mB0);
                    tc::tmap_acquire(&st->mB1);
                    seen = si;
                }
                const int local = item - st->item0, nM = st->nM, NCH = st->NCH;
                const int k = local / nM, m = local - k * nM;
                for (int ch = 0; ch < NCH; ++ch, ++g) {
                    const int stg = (int)(g % nst);
                    if (g >= nst && !tc::mbar_wait(&empty[stg], (uint32_t)(((g / nst) - 1) & 1), wb)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sb = sm + (size_t)stg * st_bytes;
                    // the stage holds BNmax rows of B; this stack's box fills BN of them
                    tc::mbar_arrive_expect_tx(&full[stg], NPA * a_bytes + NPB * (uint32_t)st->BN * 128u);
                    // A planes are read once (evict first); the radial table
                    // B is read by every item of its k (normal)
                    const unsigned long long pf = l2_evict_first();
                    tc::tma_load_3d_hint(sb, &st->mA0, &full[stg], ch * KCH, 128 * m, k, pf);
                    if (NPA > 1) tc::tma_load_3d_hint(sb + a_bytes, &st->mA1, &full[stg], ch * KCH, 128 * m, k, pf);
                    tc::tma_load_3d(sb + NPA * a_bytes, &st->mB0, &full[stg], ch * KCH, 0, k);
                    if (NPB > 1) tc::tma_load_3d(sb + NPA * a_bytes + b_bytes, &st->mB1, &full[stg], ch * KCH, 0, k);
                }
            }
            if (!ok) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
            }
            // every issued copy lands before the CTA may leave
            for (int64_t h = (g > nst ? g - nst : 0); h < g; ++h)
                tc::mbar_wait(&full[h % nst], (uint32_t)((h / nst) & 1), TC_BUDGET);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                  // ---- MMA issue
            int64_t g = 0;
            bool ok = true;
            int it = 0;
            int si = 0;
            // p_k and the K chunks of the next item are loaded one item ahead,
            // off the MMA stream
            int pk_next = 0, nch_next = 0;
            if (myitems > 0) {
                const TcStack *st = tc_stack_of<GROUP>(one, many, S, blockIdx.x, si);
                pk_next = __ldg(&st->pk[(blockIdx.x - st->item0) / st->nM]);
                nch_next = st->NCH;
            }
            for (; it < myitems && ok; ++it) {
                const int pk = pk_next, NCH = nch_next;
                if (it + 1 < myitems) {
                    const int item1 = blockIdx.x + (it + 1) * gridDim.x;
                    const TcStack *st = tc_stack_of<GROUP>(one, many, S, item1, si);
                    pk_next = __ldg(&st->pk[(item1 - st->item0) / st->nM]);
                    nch_next = st->NCH;
                }
                const int BN = max(16, (pk + 15) & ~15);
                const uint32_t id = tc::idesc(KIND == 0 ? 2 : 1, 128, BN);
                const int a = it & 1;
                if (it >= 2 && !tc::mbar_wait(&acce[a], (uint32_t)(((it >> 1) - 1) & 1), wb)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dt = tbase + (uint32_t)(a * acc_cols);
                for (int ch = 0; ch < NCH; ++ch, ++g) {
                    const int stg = (int)(g % nst);
                    if (!tc::mbar_wait(&full[stg], (uint32_t)((g / nst) & 1), wb)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(sm + (size_t)stg * st_bytes);
#pragma unroll
                    for (int pr = 0; pr < NPROD; ++pr) {
                        const int pa = (pr == 2) ? 1 : 0;   // products (0,0), (0,1), (1,0)
                        const int pb = (pr == 1) ? 1 : 0;
                        const uint32_t a0 = sa + pa * a_bytes;
                        const uint32_t b0 = sa + NPA * a_bytes + pb * b_bytes;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = tc::desc_sw128(a0 + 32u * ks);
                            const uint64_t bd = tc::desc_sw128(b0 + 32u * ks);
                            const uint32_t accf_ = (ch > 0 || pr > 0 || ks > 0) ? 1u : 0u;
                            if (KIND == 0) tc::mma_tf32(dt, ad, bd, id, accf_);
                            else tc::mma_bf16(dt, ad, bd, id, accf_);
                        }
                    }
                    tc::mma_commit(&empty[stg]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[a]);
            }
            if (!ok) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
                tc::mma_commit(&accf[it & 1]);   // tracks every MMA issued so far
                tc::mbar_wait(&accf[it & 1], (uint32_t)((it >> 1) & 1), TC_BUDGET);
            }
        }
    } else {                                              // ---- epilogue warps
        const int q4 = warp & 3;                          // TMEM lanes 32 q4 .. 32 q4 + 31
        const int cg = (warp - 2) >> 2;                   // which column groups of 16
        const int r = 32 * q4 + lane;                     // accumulator row: image r/2, part r%2
        const int et = threadIdx.x - 64;                  // 0 .. 32 TCB_EPI - 1
        int si = 0;
        for (int it = 0; it < myitems; ++it) {
            const int item = blockIdx.x + it * gridDim.x;
            const TcStack *st = tc_stack_of<GROUP>(one, many, S, item, si);
            const int local = item - st->item0, nM = st->nM;
            const int k = local / nM, m = local - k * nM;
            const int pk = __ldg(&st->pk[k]), o = __ldg(&st->off[k]);
            const int BN = max(16, (pk + 15) & ~15);
            const int a = it & 1;
            // after a failure elsewhere, stop waiting long (the loop count stays
            // the same for all epilogue warps: they meet at named barriers)
            const bool live = *(volatile int *)okflag != 0;
            const bool ok = tc::mbar_wait(&accf[a], (uint32_t)((it >> 1) & 1), live ? wb : 0);
            if (!ok && live) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
            }
            tc::fence_after_sync();
            if (ok) {
                for (int c16 = 16 * cg; c16 < BN; c16 += 16 * (TCB_EPI / 4)) {
                    float v[16];
                    tc::tmem_ld16(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(a * acc_cols + c16), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) stage[(r >> 1) * ldst + 2 * (c16 + i) + (r & 1)] = v[i];
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);
            epi_bar();                                    // the stage holds the item
            if (ok) {
                const int i0 = 64 * m;
                const int nimg_t = min(64, st->nimg - i0);
                const int P = st->P;
                float2 *out = (float2 *)st->coef;
                // t / pk as a multiply-high (exact for t < 2^32 / pk); pk = 1
                // would overflow the multiplier and is taken as is
                const unsigned magic = (pk > 1) ? 0xFFFFFFFFu / (unsigned)pk + 1u : 0u;
                for (int t = et; t < nimg_t * pk; t += 32 * TCB_EPI) {
                    const int ii = (pk > 1) ? (int)__umulhi((unsigned)t, magic) : t, q = t - ii * pk;
                    float2 val = make_float2(stage[ii * ldst + 2 * q], stage[ii * ldst + 2 * q + 1]);
                    if (k == 0) val.y = 0.f;
                    out[(size_t)(i0 + ii) * P + o + q] = val;
                }
            }
            epi_bar();                                    // the stage may be refilled
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, (uint32_t)(2 * acc_cols));
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
    int BN = 0, tmem_cols = 0, ld = 0;
    int grp = 1;                           // chunks per quadrature launch
    void *bhi = nullptr, *blo = nullptr;   // padded radial tables [k][BN][ld]
    void *ahi = nullptr, *alo = nullptr;   // ring spectra planes [k][2 grp chunk][ld]
    TcStack one;                           // maps and plan fields of this plan's launches
    // ring DFT on the tensor cores (ffb_tc_dft_*): its tables and stack
    void *dft_hi = nullptr, *dft_lo = nullptr;
    TcStack dft;                           // its four TMA maps
    int dft_ready = 0;
};

static TcState *tc_state(ffb_plan_t p) {
    if (!p->tc) p->tc = new TcState();
    return (TcState *)p->tc;
}

void ffb_tc_release(ffb_plan_t p) {
    if (!p->tc) return;
    TcState *t = (TcState *)p->tc;
    void *ptrs[] = {t->bhi, t->blo, t->ahi, t->alo, t->dft_hi, t->dft_lo};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete t;
    p->tc = nullptr;
}

static bool is_bf16(int prec) { return prec == FFB_BF16 || prec == FFB_BF16X3; }
static bool is_x3(int prec) { return prec == FFB_BF16X3 || prec == FFB_TF32X3; }

// one pipeline stage holds every plane of one 128-byte K chunk: A (128 rows)
// and B (BN rows), hi and lo for the compensated forms
static size_t tc_stage_bytes(int prec, int BN) {
    const int np = is_x3(prec) ? 2 : 1;
    return (size_t)np * 128 * 128 + (size_t)np * BN * 128;
}

static size_t tc_smem_bytes(int prec, int BN, int nst) {
    const size_t ring = (size_t)nst * tc_stage_bytes(prec, BN);
    const size_t stage = ((size_t)64 * (2 * BN + 2) * 4 + 15) & ~(size_t)15;
    return 1024 + ring + stage + 8 * (2 * (size_t)nst + 4) + 16;
}

// stages of the K pipeline: as many as fit in one CTA's shared memory next to
// the epilogue stage, at most 4; 0 when not even one fits
static int tc_stages(int prec, int ld, int BN) {
    (void)ld;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int nst = 4;
    while (nst > 0 && tc_smem_bytes(prec, BN, nst) > (size_t)optin) --nst;
    return nst;
}

bool ffb_tc_supported(ffb_plan_t p) {
    const int es = is_bf16(p->precision) ? 2 : 4;
    const int kch = 128 / es;
    const int ld = (p->n_xi + kch - 1) / kch * kch;
    const int BN = (p->pmax + 15) & ~15;
    if (BN > 256) return false;
    return tc_stages(p->precision, ld, BN) > 0;
}

int ffb_tc_prepare(ffb_plan_t p, cudaStream_t s, RingOut *out) {
    TcState *t = tc_state(p);
    const bool bf16 = is_bf16(p->precision);
    const size_t es = bf16 ? 2 : 4;
    if (t->prepared != p->precision) {
        const int kch = (int)(128 / es);
        t->ld = (p->n_xi + kch - 1) / kch * kch;
        t->BN = (p->pmax + 15) & ~15;
        if (t->BN > 256) return FFB_ERR_UNSUPPORTED;
        t->tmem_cols = 32;
        while (t->tmem_cols < t->BN) t->tmem_cols <<= 1;
        for (void **q : {&t->bhi, &t->blo, &t->ahi, &t->alo})
            if (*q) {
                cudaFree(*q);
                *q = nullptr;
            }
        const size_t nb = (size_t)(p->k_max + 1) * t->BN * t->ld;
        // the fused path's ring FFT writes the planes of several chunks before
        // one quadrature launch takes them all (fewer, fuller launches): as
        // many as fit in FFB_PLANE_BUDGET_MB, at most 4; the separate-kernel
        // path converts one chunk
        const int np = (p->precision == FFB_TF32X3 || p->precision == FFB_BF16X3) ? 2 : 1;
        const size_t per_chunk = (size_t)(p->k_max + 1) * p->chunk * 2 * t->ld * es * np;
        t->grp = p->fused ? (int)std::max<size_t>(1, std::min<size_t>(4, ((size_t)FFB_PLANE_BUDGET_MB << 20) / per_chunk)) : 1;
        const size_t na = (size_t)(p->k_max + 1) * t->grp * p->chunk * 2 * t->ld;
        int e;
        if ((e = ffb_check_cuda(cudaMalloc(&t->bhi, nb * es)))) return e;
        if ((e = ffb_check_cuda(cudaMalloc(&t->blo, nb * es)))) return e;
        if ((e = ffb_check_cuda(cudaMalloc(&t->ahi, na * es)))) return e;
        if ((e = ffb_check_cuda(cudaMalloc(&t->alo, na * es)))) return e;
        // padding columns j >= n_xi stay zero for the whole life of the plan
        if ((e = ffb_check_cuda(cudaMemsetAsync(t->ahi, 0, na * es, s)))) return e;
        if ((e = ffb_check_cuda(cudaMemsetAsync(t->alo, 0, na * es, s)))) return e;
        const unsigned g = (unsigned)((nb + 255) / 256);
        if (bf16)
            k_prep_bpad<true><<<g, 256, 0, s>>>(p->d_B64, p->d_p, p->d_off, p->k_max, t->BN, p->n_xi, t->ld,
                                                t->bhi, t->blo);
        else
            k_prep_bpad<false><<<g, 256, 0, s>>>(p->d_B64, p->d_p, p->d_off, p->k_max, t->BN, p->n_xi, t->ld,
                                                 t->bhi, t->blo);
        p->launches++;
        if ((e = ffb_check_cuda(cudaGetLastError()))) return e;
        const uint64_t rows = 2ull * t->grp * p->chunk;
        TcStack &o = t->one;
        std::memset(&o, 0, sizeof o);
        if ((e = make_map(&o.mA0, t->ahi, bf16, t->ld, rows, p->k_max + 1, 128))) return e;
        if ((e = make_map(&o.mA1, t->alo, bf16, t->ld, rows, p->k_max + 1, 128))) return e;
        if ((e = make_map(&o.mB0, t->bhi, bf16, t->ld, t->BN, p->k_max + 1, t->BN))) return e;
        if ((e = make_map(&o.mB1, t->blo, bf16, t->ld, t->BN, p->k_max + 1, t->BN))) return e;
        o.pk = p->d_p;
        o.off = p->d_off;
        o.P = p->P;
        o.NCH = t->ld / kch;
        o.BN = t->BN;
        t->prepared = p->precision;
    }
    if (out) {
        switch (p->precision) {
            case FFB_TF32: out->fmt = FFB_FMT_TF32; break;
            case FFB_TF32X3: out->fmt = FFB_FMT_TF32X2; break;
            case FFB_BF16: out->fmt = FFB_FMT_BF16; break;
            default: out->fmt = FFB_FMT_BF16X2; break;
        }
        out->p0 = t->ahi;
        out->p1 = t->alo;
        out->ld = t->ld;
        out->lead = t->grp * p->chunk;
    }
    return FFB_OK;
}

int ffb_tc_group(ffb_plan_t p) { return p->tc ? ((TcState *)p->tc)->grp : 1; }

// launch shape of the quadrature: two CTAs per SM when a two-stage ring fits
// in half the shared memory (their epilogues then overlap each other's
// loads), else one with the deepest ring that fits
static void tc_launch_shape(int prec, int BN, int *per_sm, int *nst) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    *per_sm = 1;
    *nst = tc_stages(prec, 0, BN);
    if (*nst > 0 && 2 * tc_smem_bytes(prec, BN, 2) + 2048 <= (size_t)optin) {
        *per_sm = 2;
        *nst = 2;
    }
}

template <int KIND, int NPA, int NPB, int NPROD, bool GROUP>
static int launch_tc_kernel(int prec, const TcStack &one, const TcStack *many, int S, int nitems, int BNmax,
                            int acc_cols, int per_sm, int nst, int *status, long long wb, cudaStream_t s) {
    if (nst <= 0 || nitems <= 0) return nitems <= 0 ? FFB_OK : FFB_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = tc_smem_bytes(prec, BNmax, nst);
    static int attr = 0;
    if (attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_tc_bessel<KIND, NPA, NPB, NPROD, GROUP>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    const int grid = nitems < per_sm * sms ? nitems : per_sm * sms;   // persistent CTAs
    // launched with programmatic serialization: the prologue (barriers, TMEM)
    // overlaps the previous kernel's tail; the producer waits before its loads
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * TCB_WARPS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {ffb_pdl_attr()};
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return ffb_check_cuda(cudaLaunchKernelEx(&cfg, k_tc_bessel<KIND, NPA, NPB, NPROD, GROUP>, one, many, S, BNmax,
                                             acc_cols, nst, nitems, status, wb));
}

template <bool GROUP>
static int launch_tc_prec(int prec, const TcStack &one, const TcStack *many, int S, int nitems, int BNmax,
                          int acc_cols, int per_sm, int nst, int *status, long long wb, cudaStream_t s) {
    switch (prec) {
        case FFB_TF32: return launch_tc_kernel<0, 1, 1, 1, GROUP>(prec, one, many, S, nitems, BNmax, acc_cols, per_sm, nst, status, wb, s);
        case FFB_TF32X3: return launch_tc_kernel<0, 2, 2, 3, GROUP>(prec, one, many, S, nitems, BNmax, acc_cols, per_sm, nst, status, wb, s);
        case FFB_BF16: return launch_tc_kernel<1, 1, 1, 1, GROUP>(prec, one, many, S, nitems, BNmax, acc_cols, per_sm, nst, status, wb, s);
        case FFB_BF16X3: return launch_tc_kernel<1, 2, 2, 3, GROUP>(prec, one, many, S, nitems, BNmax, acc_cols, per_sm, nst, status, wb, s);
        default: return FFB_ERR_ARG;
    }
}

static int launch_tc(ffb_plan_t p, TcState *t, int nimg, float *d_coef_chunk, cudaStream_t s) {
    int per_sm = 1, nst = 0;
    tc_launch_shape(p->precision, t->BN, &per_sm, &nst);
    if (nst <= 0) return FFB_ERR_UNSUPPORTED;
    TcStack one = t->one;
    one.coef = d_coef_chunk;
    one.nimg = nimg;
    one.nM = (2 * nimg + 127) / 128;
    one.item0 = 0;
    const int nitems = one.nM * (p->k_max + 1);
    ProfScope ps(p, FFB_KC_BESSEL, s);
    const int e = launch_tc_prec<false>(p->precision, one, nullptr, 1, nitems, t->BN, t->tmem_cols, per_sm, nst,
                                        p->d_status, p->wait_budget, s);
    p->launches++;
    return e;
}

// ---------------------------------------------------------------------------
// Ring DFT on the tensor cores (Eq. 1DFFT at n_theta = 512, BF16x3, the
// shared-memory grid path with 128 rings per image).  With the conjugate
// completion f_{l + n/2} = conj f_l of a ring, f = u + i v,
//   F_k = s sum_{l < n/2} e^{-i k theta_l} (f_l + (-1)^k conj f_l),  s = 2 pi / n,
// i.e. F_k = 2 s sum_l u_l e^{-i k theta_l} for even k and
// F_k = 2 s sum_l v_l (sin k theta_l + i cos k theta_l) for odd k: two real
// contractions over l, of the rings' real parts with the even-k table and of
// their imaginary parts with the odd-k table, 192 columns (re, im of 96 k)
// each.  The grid kernel leaves u and v as bf16 hi / lo planes
// [hi, lo][u, v][image][ring][l] in the polar buffer.  CTA b of a launch
// takes the parity p = b mod 2 (with 96-column slices also the half
// (b / 2) mod 2, its slice resident in shared memory) and the images
// b / NGRP, b / NGRP + G / NGRP, ...; one image (its 128 rings) is one M
// tile, K = 256 in four 128-byte chunks streamed by TMA (with the table's
// chunk beside it when it streams).  BF16x3: A_hi B_hi + A_hi B_lo + A_lo B_hi
// into one of two TMEM accumulators; eight epilogue warps write the spectra
// as the quadrature's operand planes (bf16 hi / lo, [k][image][re, im][ring],
// 32 rings per warp store).  This trades the FFT's 1.5 MFLOP per image for
// 2 x 3 x 128 x 192 x 256 x 2 = 75.5 MFLOP on the tensor cores.
// Waits are bounded like the quadrature's.  Measured at L = 128 (per 100k
// images): the register FFT 16.9 ms, this kernel 12.5 ms with resident
// 96-column slices and 12.0 ms with the streamed 192-column table; the
// timeline of the 96-column form (clock64 stamps) shows one image's 48 MMAs
// (M 128 x N 96 x K 16) taking about 5.4 k cycles with or without the ring
// loads, about half the tensor cores' dense rate, the epilogue (3.1 k
// cycles) overlapping them.
// ---------------------------------------------------------------------------
#define TC_DFT_BN 192            // table columns per parity
// columns per CTA: all 192, the table streamed beside the rings through two
// 80 KB stages (48 MMAs of N = 192 per image and parity), or 96, half a
// table kept in shared memory and the rings through four 32 KB stages
// (measured per 100k images at L = 128: 12.0 ms and 12.5 ms)
#ifndef TC_DFT_NB
#define TC_DFT_NB 192
#endif
#define TC_DFT_RES (TC_DFT_NB < TC_DFT_BN)                // the CTA's table slice stays in shared memory
#define TC_DFT_NGRP (2 * TC_DFT_BN / TC_DFT_NB)           // CTAs per image: parities x column slices
#define TC_DFT_NST (TC_DFT_RES ? 4 : 2)                   // pipeline stages
#define TC_DFT_A_BYTES (2u * 128u * 128u)              // one K chunk of an image's rings: hi and lo, 128 rows x 128 B
#define TC_DFT_B_BYTES (2u * TC_DFT_NB * 128u)         // one K chunk of the table slice: hi and lo
#define TC_DFT_STAGE (TC_DFT_A_BYTES + (TC_DFT_RES ? 0u : TC_DFT_B_BYTES))
#define TC_DFT_NCH 4             // 128-byte K chunks (K = 256 bf16)

static size_t tc_dft_smem() {
    return 1024 + (TC_DFT_RES ? (size_t)TC_DFT_NCH * TC_DFT_B_BYTES : 0) + (size_t)TC_DFT_NST * TC_DFT_STAGE +
           8 * (2 * TC_DFT_NST + 5) + 16;
}

__global__ void __launch_bounds__(32 * TCB_WARPS)
k_tc_ringdft(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
             const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
             __nv_bfloat16 *__restrict__ out0, __nv_bfloat16 *__restrict__ out1, int lead, int ld, int kmax,
             int nimg, int nring, int *status, long long wb) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *bsm = sm;                                              // [NCH][hi, lo][96 rows][128 B]
    uint8_t *asm_ = sm + (TC_DFT_RES ? TC_DFT_NCH * TC_DFT_B_BYTES : 0);   // [NST] stages
    uint64_t *bars = (uint64_t *)(asm_ + TC_DFT_NST * TC_DFT_STAGE);
    uint64_t *full = bars, *empty = bars + TC_DFT_NST, *accf = bars + 2 * TC_DFT_NST,
             *acce = bars + 2 * TC_DFT_NST + 2, *bfull = bars + 2 * TC_DFT_NST + 4;
    uint32_t *slot = (uint32_t *)(bars + 2 * TC_DFT_NST + 5);
    int *okflag = (int *)(slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int par = blockIdx.x & 1, hcol = TC_DFT_RES ? (blockIdx.x >> 1) & 1 : 0;
    const int step = gridDim.x / TC_DFT_NGRP;
    const int first = blockIdx.x / TC_DFT_NGRP;
    const int myitems = (first < nimg) ? (nimg - 1 - first) / step + 1 : 0;
    constexpr int ACC = TC_DFT_NB <= 128 ? 128 : 256;               // TMEM columns per accumulator
    pdl_trigger();

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * TC_DFT_NST; ++i) tc::mbar_init(&bars[i], 1);
        tc::mbar_init(&accf[0], 1);
        tc::mbar_init(&accf[1], 1);
        tc::mbar_init(&acce[0], TCB_EPI);
        tc::mbar_init(&acce[1], TCB_EPI);
        tc::mbar_init(bfull, 1);
        tc::fence_mbar_init();
        *okflag = 1;
    }
    if (warp == 1) {
        tc::tmem_alloc(slot, 2 * ACC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;

    if (warp == 0) {
        if (lane == 0) {                                  // ---- TMA producer
            pdl_wait();   // the polar planes come from the grid kernel
            // the CTA's table slice, once: rows hcol * 96 .. + 95 of parity par
            if (TC_DFT_RES) {
                tc::mbar_arrive_expect_tx(bfull, TC_DFT_NCH * TC_DFT_B_BYTES);
                for (int ch = 0; ch < TC_DFT_NCH; ++ch) {
                    uint8_t *b = bsm + ch * TC_DFT_B_BYTES;
                    tc::tma_load_3d(b, &mB0, bfull, ch * 64, hcol * TC_DFT_NB, par);
                    tc::tma_load_3d(b + TC_DFT_B_BYTES / 2, &mB1, bfull, ch * 64, hcol * TC_DFT_NB, par);
                }
            }
            const unsigned long long pf = l2_evict_first();
            int64_t g = 0;
            bool ok = true;
            for (int it = 0; it < myitems && ok && *(volatile int *)okflag; ++it) {
                const int img = first + it * step;
                for (int ch = 0; ch < TC_DFT_NCH; ++ch, ++g) {
                    const int stg = (int)(g % TC_DFT_NST);
                    if (g >= TC_DFT_NST &&
                        !tc::mbar_wait(&empty[stg], (uint32_t)(((g / TC_DFT_NST) - 1) & 1), wb)) {
                        ok = false;
                        break;
                    }
                    uint8_t *a = asm_ + stg * TC_DFT_STAGE;
                    tc::mbar_arrive_expect_tx(&full[stg], TC_DFT_STAGE);
                    tc::tma_load_3d_hint(a, &mA0, &full[stg], ch * 64, 128 * img, par, pf);
                    tc::tma_load_3d_hint(a + TC_DFT_A_BYTES / 2, &mA1, &full[stg], ch * 64, 128 * img, par, pf);
                    if (!TC_DFT_RES) {   // the table's K chunk beside the rings' (streamed)
                        uint8_t *b = a + TC_DFT_A_BYTES;
                        tc::tma_load_3d(b, &mB0, &full[stg], ch * 64, 0, par);
                        tc::tma_load_3d(b + TC_DFT_B_BYTES / 2, &mB1, &full[stg], ch * 64, 0, par);
                    }
                }
            }
            if (!ok) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
            }
            // every issued copy lands before the CTA may leave
            if (TC_DFT_RES) tc::mbar_wait(bfull, 0u, TC_BUDGET);
            for (int64_t h = (g > TC_DFT_NST ? g - TC_DFT_NST : 0); h < g; ++h)
                tc::mbar_wait(&full[h % TC_DFT_NST], (uint32_t)((h / TC_DFT_NST) & 1), TC_BUDGET);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                  // ---- MMA issue
            int64_t g = 0;
            bool ok = TC_DFT_RES ? tc::mbar_wait(bfull, 0u, wb) : true;
            int it = 0;
            const uint32_t id = tc::idesc(1, 128, TC_DFT_NB);
            for (; it < myitems && ok; ++it) {
                const int a = it & 1;
                if (it >= 2 && !tc::mbar_wait(&acce[a], (uint32_t)(((it >> 1) - 1) & 1), wb)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dt = tbase + (uint32_t)(a * ACC);
                for (int ch = 0; ch < TC_DFT_NCH; ++ch, ++g) {
                    const int stg = (int)(g % TC_DFT_NST);
                    if (!tc::mbar_wait(&full[stg], (uint32_t)((g / TC_DFT_NST) & 1), wb)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(asm_ + stg * TC_DFT_STAGE);
                    const uint32_t sb = TC_DFT_RES ? tc::smem_u32(bsm + ch * TC_DFT_B_BYTES) : sa + TC_DFT_A_BYTES;
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr) {
                        const int pa = (pr == 2) ? 1 : 0;   // products (hi, hi), (hi, lo), (lo, hi)
                        const int pb = (pr == 1) ? 1 : 0;
                        const uint32_t a0 = sa + pa * (TC_DFT_A_BYTES / 2);
                        const uint32_t b0 = sb + pb * (TC_DFT_B_BYTES / 2);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = tc::desc_sw128(a0 + 32u * ks);
                            const uint64_t bd = tc::desc_sw128(b0 + 32u * ks);
                            tc::mma_bf16(dt, ad, bd, id, (ch > 0 || pr > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&empty[stg]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[a]);
            }
            if (!ok) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
                tc::mma_commit(&accf[it & 1]);   // tracks every MMA issued so far
                tc::mbar_wait(&accf[it & 1], (uint32_t)((it >> 1) & 1), TC_BUDGET);
            }
        }
    } else {                                              // ---- epilogue warps
        // accumulator row = ring j of the item's image, column c of the
        // slice = table column hcol * 96 + c: spectrum F_kk, kk = 2 (col / 2)
        // + par, part col mod 2
        const int q4 = warp & 3;
        const int cg = (warp - 2) >> 2;
        const int j = 32 * q4 + lane;
        for (int it = 0; it < myitems; ++it) {
            const int img = first + it * step;
            const int a = it & 1;
            const bool live = *(volatile int *)okflag != 0;
            const bool ok = tc::mbar_wait(&accf[a], (uint32_t)((it >> 1) & 1), live ? wb : 0);
            if (!ok && live) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
            }
            tc::fence_after_sync();
            if (ok) {
                // columns 2e, 2e + 1 of the slice are re, im of k = col0 + 2e + par
                // (col0 even): plane offsets k S + (2 img) ld + j and that + ld,
                // S = 2 lead ld (32-bit: the group's planes hold < 2^31 values)
                const int S = 2 * lead * ld;
                const int base = 2 * img * ld + j;
                for (int c16 = 16 * cg; c16 < TC_DFT_NB; c16 += 16 * (TCB_EPI / 4)) {
                    float v[16];
                    tc::tmem_ld16(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(a * ACC + c16), v);
                    const int k0 = hcol * TC_DFT_NB + c16 + par;
                    const int o0 = k0 * S + base;
                    if (j < nring) {
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            if (k0 + i <= kmax) {
                                const int o = o0 + i * S;
                                const __nv_bfloat16 hr = __float2bfloat16_rn(v[i]);
                                const __nv_bfloat16 hi_ = __float2bfloat16_rn(v[i + 1]);
                                out0[o] = hr;
                                out1[o] = __float2bfloat16_rn(v[i] - __bfloat162float(hr));
                                out0[o + ld] = hi_;
                                out1[o + ld] = __float2bfloat16_rn(v[i + 1] - __bfloat162float(hi_));
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, 2 * ACC);
}

bool ffb_tc_dft_ok(ffb_plan_t p) {
    return p->fused && p->precision == FFB_BF16X3 && p->n_theta == 512 && p->n_xi == 128 &&
           2 * (p->k_max / 2 + 1) <= TC_DFT_BN;
}

// the ring DFT's tables [parity][192 columns][n/2] as bf16 hi / lo: column
// 2e + c of parity p is part c (re, im) of k = 2e + p; zero for k > k_max
static int tc_dft_table(int n, int kmax, std::vector<__nv_bfloat16> &hi, std::vector<__nv_bfloat16> &lo) {
    if (n < 4 || (n & 1) || kmax < 0 || 2 * (kmax / 2 + 1) > TC_DFT_BN) return FFB_ERR_UNSUPPORTED;
    const int nh = n / 2, BN = TC_DFT_BN;
    const double sc = 2.0 * (2.0 * M_PI / (double)n);
    hi.assign((size_t)2 * BN * nh, __float2bfloat16_rn(0.f));
    lo.assign((size_t)2 * BN * nh, __float2bfloat16_rn(0.f));
    for (int par = 0; par < 2; ++par)
        for (int col = 0; col < BN; ++col) {
            const int k = 2 * (col >> 1) + par, c = col & 1;
            if (k > kmax) continue;
            for (int l = 0; l < nh; ++l) {
                const double a = 2.0 * M_PI * (double)(((long long)k * l) % n) / (double)n;
                const double v = (par == 0) ? (c ? -sc * std::sin(a) : sc * std::cos(a))
                                            : (c ? sc * std::cos(a) : sc * std::sin(a));
                const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                const size_t i = ((size_t)par * BN + col) * nh + l;
                hi[i] = h;
                lo[i] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
            }
        }
    return FFB_OK;
}

extern "C" int ffb_ringdft_table(int n_theta, int k_max, float *h_hi, float *h_lo) {
    std::vector<__nv_bfloat16> hi, lo;
    const int e = tc_dft_table(n_theta, k_max, hi, lo);
    if (e) return e;
    for (size_t i = 0; i < hi.size(); ++i) {
        if (h_hi) h_hi[i] = __bfloat162float(hi[i]);
        if (h_lo) h_lo[i] = __bfloat162float(lo[i]);
    }
    return FFB_OK;
}

int ffb_tc_dft_prepare(ffb_plan_t p, cudaStream_t s) {
    TcState *t = tc_state(p);
    if (t->dft_ready) return FFB_OK;
    if (!ffb_tc_dft_ok(p) || !p->d_Fpol) return FFB_ERR_UNSUPPORTED;
    const int n = p->n_theta, nh = n / 2, BN = TC_DFT_BN;
    std::vector<__nv_bfloat16> hi, lo;
    int e = tc_dft_table(n, p->k_max, hi, lo);
    if (e) return e;
    const size_t tb = sizeof(__nv_bfloat16) * hi.size();
    if ((e = ffb_check_cuda(cudaMalloc(&t->dft_hi, tb)))) return e;
    if ((e = ffb_check_cuda(cudaMalloc(&t->dft_lo, tb)))) return e;
    if ((e = ffb_check_cuda(cudaMemcpyAsync(t->dft_hi, hi.data(), tb, cudaMemcpyHostToDevice, s)))) return e;
    if ((e = ffb_check_cuda(cudaMemcpyAsync(t->dft_lo, lo.data(), tb, cudaMemcpyHostToDevice, s)))) return e;
    if ((e = ffb_check_cuda(cudaStreamSynchronize(s)))) return e;
    // A: the polar buffer as four bf16 planes of chunk x n_xi rows of nh
    const uint64_t rows = (uint64_t)p->chunk * p->n_xi;
    __nv_bfloat16 *pl = (__nv_bfloat16 *)p->d_Fpol;
    TcStack &d = t->dft;
    std::memset(&d, 0, sizeof d);
    if ((e = make_map(&d.mA0, pl, true, nh, rows, 2, 128))) return e;
    if ((e = make_map(&d.mA1, pl + 2 * rows * nh, true, nh, rows, 2, 128))) return e;
    if ((e = make_map(&d.mB0, t->dft_hi, true, nh, BN, 2, TC_DFT_NB))) return e;
    if ((e = make_map(&d.mB1, t->dft_lo, true, nh, BN, 2, TC_DFT_NB))) return e;
    t->dft_ready = 1;
    return FFB_OK;
}

// one launch per chunk of m images: F of every ring into the operand planes
// of the group (r: the chunk's first image in them)
int ffb_launch_tc_dft(ffb_plan_t p, int m, const RingOut &r, cudaStream_t s) {
    int e = ffb_tc_dft_prepare(p, s);
    if (e) return e;
    if (m <= 0) return FFB_OK;
    TcState *t = tc_state(p);
    const size_t smem = tc_dft_smem();
    static int attr = 0;
    if (attr < (int)smem) {
        if ((e = ffb_check_cuda(cudaFuncSetAttribute(k_tc_ringdft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem))))
            return e;
        attr = (int)smem;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int grid = TC_DFT_NGRP * std::max(1, std::min(sms / TC_DFT_NGRP, m));   // (parity, slice) x image groups
    ProfScope ps(p, FFB_KC_RING_FFT, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * TCB_WARPS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {ffb_pdl_attr()};
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = ffb_check_cuda(cudaLaunchKernelEx(&cfg, k_tc_ringdft, t->dft.mA0, t->dft.mA1, t->dft.mB0, t->dft.mB1,
                                          (__nv_bfloat16 *)r.p0, (__nv_bfloat16 *)r.p1, r.lead, r.ld, p->k_max, m,
                                          p->n_xi, p->d_status, p->wait_budget));
    p->launches++;
    return e;
}

// the separate-kernel path's float32 ring spectra of one chunk -> the
// operand planes of the tensor-core quadrature
int ffb_tc_split_planes(ffb_plan_t p, cudaStream_t s) {
    int e = ffb_tc_prepare(p, s, nullptr);
    if (e) return e;
    TcState *t = tc_state(p);
    {
        const int64_t total = (int64_t)(p->k_max + 1) * p->chunk * 2 * p->n_xi;
        const unsigned g = (unsigned)((total + 255) / 256);
        ProfScope ps(p, FFB_KC_BESSEL, s);
        switch (p->precision) {
            case FFB_TF32: k_split_planes<false, false><<<g, 256, 0, s>>>(p->d_Fhat, total, p->n_xi, t->ld, t->ahi, t->alo); break;
            case FFB_TF32X3: k_split_planes<false, true><<<g, 256, 0, s>>>(p->d_Fhat, total, p->n_xi, t->ld, t->ahi, t->alo); break;
            case FFB_BF16: k_split_planes<true, false><<<g, 256, 0, s>>>(p->d_Fhat, total, p->n_xi, t->ld, t->ahi, t->alo); break;
            default: k_split_planes<true, true><<<g, 256, 0, s>>>(p->d_Fhat, total, p->n_xi, t->ld, t->ahi, t->alo); break;
        }
        p->launches++;
        if ((e = ffb_check_cuda(cudaGetLastError()))) return e;
    }
    return FFB_OK;
}

int ffb_launch_bessel_tc(ffb_plan_t p, int nimg, float *d_coef_chunk, bool planes_ready, cudaStream_t s) {
    int e = ffb_tc_prepare(p, s, nullptr);
    if (e) return e;
    if (!planes_ready && (e = ffb_tc_split_planes(p, s))) return e;
    return launch_tc(p, tc_state(p), nimg, d_coef_chunk, s);
}

// ---- grouped quadrature: the (stack, k, M tile) items of several plans in
// one launch, the stacks' descriptors in device memory
size_t ffb_tc_stack_bytes() { return sizeof(TcStack); }

int ffb_tc_bn(ffb_plan_t p) { return p->tc ? ((TcState *)p->tc)->BN : 0; }

// stack descriptor of plan p for nimg images whose coefficients start at
// coef, its items numbered from item0 (host memory at dst); returns the
// stack's item count through *nitems
int ffb_tc_stack_fill(ffb_plan_t p, float *coef, int nimg, int item0, void *dst, int *nitems) {
    if (!p->tc || ((TcState *)p->tc)->prepared != p->precision) return FFB_ERR_STATE;
    TcStack st = ((TcState *)p->tc)->one;
    st.coef = coef;
    st.nimg = nimg;
    st.nM = (2 * nimg + 127) / 128;
    st.item0 = item0;
    std::memcpy(dst, &st, sizeof st);
    *nitems = st.nM * (p->k_max + 1);
    return FFB_OK;
}

// launch shapes the group's tuner may time for stacks of width BNmax:
// (CTAs per SM, pipeline stages); returns the count written (at most 4)
int ffb_tc_group_shapes(int prec, int BNmax, int *per_sm, int *nst) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int deep = tc_stages(prec, 0, BNmax);
    int n = 0;
    for (int st = deep; st >= 2 && n < 3; --st) {
        per_sm[n] = 1;
        nst[n++] = st;
    }
    if (deep >= 2 && 2 * tc_smem_bytes(prec, BNmax, 2) + 2048 <= (size_t)optin) {
        per_sm[n] = 2;
        nst[n++] = 2;
    }
    if (n == 0 && deep == 1) {
        per_sm[0] = 1;
        nst[0] = 1;
        n = 1;
    }
    return n;
}

int ffb_tc_group_bessel(int prec, const void *d_stacks, int S, int nitems, int BNmax, int per_sm, int nst,
                        int *status, long long wb, cudaStream_t s) {
    if (S <= 0 || nitems <= 0) return FFB_OK;
    int acc_cols = 32;
    while (acc_cols < BNmax) acc_cols <<= 1;
    TcStack none;
    std::memset(&none, 0, sizeof none);
    return launch_tc_prec<true>(prec, none, (const TcStack *)d_stacks, S, nitems, BNmax, acc_cols, per_sm, nst,
                                status, wb, s);
}

// ---------------------------------------------------------------------------
// a6/a7 on the tensor cores: C^(k) += X X^T, X = [Re A^(k), Im A^(k)] with rows
// q and K = (image, re/im).  Consecutive k whose block sizes sum to at most
// 128 form a super-block (the plan's table: first k, end k, first coefficient
// index, rows): its rows are the contiguous coefficient range of those k, so
// one M = 128, N = rows chain of MMAs over the super-block's X computes every
// C^(k) of it at once as the diagonal blocks of X X^T (the cross terms between
// different k are formed and never read).  At L = 128 that is 38 chains per
// image instead of 183 (the MMA issue rate bounded the per-k form).
//
// A persistent CTA walks the items (stack, super-block, image range).  For
// each item it stages tiles of 32 images from the coefficient array (one
// contiguous run of <= 128 values per image) into the 128-byte-swizzle
// K-major layout (hi/lo split, the k = 0 rows shifted by the pilot mean and
// their imaginary column zero, and summed per row for the k = 0 mean); the
// raw values arrive by cp.async in a ring
// COV_RS - 1 tiles ahead.  Tile t of an item accumulates into TMEM
// accumulator t mod nacc (4 x 128 columns): the tensor core's float32
// accumulation error grows with the number of accumulate steps, so no chain
// covers more than 128 images (items of at most 512 images); the partial
// sums are added in float32 and then to the float64 accumulator by atomics.
// ---------------------------------------------------------------------------
#define COV_NT 512   // threads of a covariance CTA
#define COV_RS 3     // tiles of coefficients in flight (shared-memory ring)
#define COV_TI 32    // images per tile
#define COV_PF 8     // slots per thread per tile: 128 rows x 32 images / 512
#define COV_NACC 4   // rotating accumulators of 128 columns

template <int KIND, int NP>
__global__ void __launch_bounds__(COV_NT, 1)
k_tc_cov(const __grid_constant__ CovGroup g, int *status, long long wb) {
    constexpr int ES = (KIND == 0) ? 4 : 2;
    constexpr int KCH = 128 / ES;               // K elements per 128-byte chunk
    constexpr int KT = 2 * COV_TI;              // K entries per tile
    constexpr int NCHT = KT / KCH;              // chunks per tile: 1 (bf16) or 2 (tf32)
    constexpr int KINST = (KIND == 0) ? 8 : 16; // K per MMA instruction
    constexpr uint32_t CH_BYTES = 128u * 128u;  // one chunk of 128 rows
    constexpr uint32_t BUF_BYTES = NP * NCHT * CH_BYTES;
    static_assert(NCHT * KCH == KT, "whole chunks per tile");
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    // per-thread ring of raw coefficient slots (each thread reads back only
    // its own slots)
    float2 *raw = (float2 *)(sm + 2 * BUF_BYTES);
    uint64_t *bars = (uint64_t *)(sm + 2 * BUF_BYTES + (size_t)COV_RS * COV_NT * COV_PF * sizeof(float2));
    uint32_t *slot = (uint32_t *)(bars + 4);
    int *okflag = (int *)(slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (uint32_t i = threadIdx.x; i < 2 * BUF_BYTES / 16; i += COV_NT)
        ((uint4 *)sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
        *okflag = 1;
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 512u);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;
    int64_t gt = 0;   // tiles committed by this CTA: buffer gt & 1, mbarrier phase (gt >> 1) & 1
    int64_t last_commit = -1;   // thread 0: the tile of the newest commit

    for (int64_t item = blockIdx.x; item < g.nitems && *okflag; item += gridDim.x) {
        const CovStack &S = g.st[cov_stack_of(g, item)];
        const int64_t local = item - S.item0;
        const int4 sb = S.work[local % S.nk];       // (first k, end k, first index, rows)
        const int64_t ib = (local / S.nk) * (int64_t)S.per;
        const int64_t ie = min(S.n, ib + (int64_t)S.per);
        const int rows = sb.w, row0 = sb.z;
        const int p0 = (sb.x == 0) ? S.pk[0] : 0;   // rows of k = 0 (shifted, real)
        const int BN = max(16, (rows + 15) & ~15);
        // (image, row) slots of a tile: each warp covers 8 rows x 4 images,
        // so that its stores into the swizzled K-major tile fall on distinct
        // banks; QBP 8-row blocks (a power of two >= rows/8) index by shifts
        int lgQ = 0;
        while ((8 << lgQ) < rows) ++lgQ;
        const int QBP = 1 << lgQ;
        const int nslots = 8 * QBP * COV_TI;
        const int ntiles = (ie > ib) ? (int)((ie - ib + COV_TI - 1) / COV_TI) : 0;
        if (nslots > COV_NT * COV_PF || rows > 128) {   // uniform across the CTA
            if (threadIdx.x == 0) ffb_flag(status, FFB_ERR_UNSUPPORTED);
            continue;
        }
        const uint32_t id = tc::idesc(KIND == 0 ? 2 : 1, 128, BN);
        const float2 *coef = S.coef + row0;
        const int P = S.P;

        // one commit group per tile (empty past the last one), so that
        // "all but the newest COV_RS - 1 groups complete" means tile t landed
        auto issue_tile = [&](int t) {
            if (t < ntiles) {
                const int64_t i0 = ib + (int64_t)t * COV_TI;
                float2 *st = raw + (size_t)(t % COV_RS) * COV_NT * COV_PF;
#pragma unroll
                for (int u = 0; u < COV_PF; ++u) {
                    const int it = threadIdx.x + COV_NT * u;
                    if (it < nslots) {
                        const int pr = it >> 5, q = 8 * (pr & (QBP - 1)) + (it & 7),
                                  ii = 4 * (pr >> lgQ) + ((it >> 3) & 3);
                        if (q < rows && i0 + ii < ie) tc::cp_async8(&st[it], &coef[(i0 + ii) * P + q]);
                        else st[it] = make_float2(0.f, 0.f);
                    }
                }
            }
            tc::cp_async_commit();
        };
#pragma unroll
        for (int t = 0; t < COV_RS - 1; ++t) issue_tile(t);
        // k = 0 rows: sums of the shifted real parts per slot (a slot keeps its
        // (row, image-in-tile) for the whole item)
        float s0acc[COV_PF];
#pragma unroll
        for (int u = 0; u < COV_PF; ++u) s0acc[u] = 0.f;
        for (int t = 0; t < ntiles; ++t, ++gt) {
            const int buf = (int)(gt & 1);
            uint8_t *B0 = sm + buf * BUF_BYTES;
            // buffer buf is free once the MMAs of tile gt - 2 are done.  A wait
            // that ran out is voted on at the tile's barrier below, so that the
            // whole CTA leaves the loop together (the tile staged meanwhile may
            // be garbage; no MMA reads it)
            const bool fail = gt >= 2 && !tc::mbar_wait(&bars[buf], (uint32_t)(((gt - 2) >> 1) & 1), wb);
            issue_tile(t + COV_RS - 1);               // COV_RS - 1 tiles stay in flight
            tc::cp_async_wait<COV_RS - 1>();
            const float2 *st = raw + (size_t)(t % COV_RS) * COV_NT * COV_PF;
            const bool last = (ib + (int64_t)(t + 1) * COV_TI > ie);
#pragma unroll
            for (int u = 0; u < COV_PF; ++u) {
                const int it = threadIdx.x + COV_NT * u;
                if (it >= nslots) break;
                const int pr = it >> 5, q = 8 * (pr & (QBP - 1)) + (it & 7), ii = 4 * (pr >> lgQ) + ((it >> 3) & 3);
                if (q >= rows) continue;   // rows past the super-block in the last 8-row block
                const float2 v = st[it];
                float re = v.x, im = v.y;
                if (q < p0) {   // k = 0: shifted real part; images past the range stay zero
                    re = (!last || ib + (int64_t)t * COV_TI + ii < ie) ? re - S.shift[q] : 0.f;
                    im = 0.f;
                    s0acc[u] += re;
                }
                const int kidx = 2 * ii;                 // K index of the real part
                const int ch = kidx / KCH, e = kidx % KCH;
                const uint32_t byte = (uint32_t)e * ES;
                const uint32_t off = ch * CH_BYTES + (q >> 3) * 1024u + (q & 7) * 128u +
                                     ((((byte >> 4) ^ (uint32_t)(q & 7)) << 4) | (byte & 15u));
                if (KIND == 0) {
                    const float rh = tf32_round(re), ih = tf32_round(im);
                    *(float2 *)(B0 + off) = make_float2(rh, ih);
                    if (NP > 1) *(float2 *)(B0 + NCHT * CH_BYTES + off) = make_float2(re - rh, im - ih);
                } else {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
                    *(__nv_bfloat162 *)(B0 + off) = h;
                    if (NP > 1) {
                        const float2 hf = __bfloat1622float2(h);
                        *(__nv_bfloat162 *)(B0 + NCHT * CH_BYTES + off) = __floats2bfloat162_rn(re - hf.x, im - hf.y);
                    }
                }
            }
            tc::fence_async_shared();   // generic-proxy writes -> visible to the tensor core
            if (__syncthreads_or(fail)) {
                if (threadIdx.x == 0) {
                    ffb_flag(status, FFB_ERR_TIMEOUT);
                    atomicExch(okflag, 0);
                }
                break;
            }
            if (threadIdx.x == 0) {
                tc::fence_after_sync();
                const uint32_t dt = tbase + (uint32_t)((t % COV_NACC) * 128);
#pragma unroll
                for (int pr = 0; pr < (NP > 1 ? 3 : 1); ++pr) {
                    const int pa = (pr == 2) ? 1 : 0, pb = (pr == 1) ? 1 : 0;
#pragma unroll
                    for (int ch = 0; ch < NCHT; ++ch) {
                        const uint32_t a0 = tc::smem_u32(B0 + (size_t)(pa * NCHT + ch) * CH_BYTES);
                        const uint32_t b0 = tc::smem_u32(B0 + (size_t)(pb * NCHT + ch) * CH_BYTES);
#pragma unroll
                        for (int ks = 0; ks < KCH / KINST; ++ks) {
                            const uint64_t ad = tc::desc_sw128(a0 + 32u * ks);
                            const uint64_t bd = tc::desc_sw128(b0 + 32u * ks);
                            const uint32_t accf = (t >= COV_NACC || pr > 0 || ch > 0 || ks > 0) ? 1u : 0u;
                            if (KIND == 0) tc::mma_tf32(dt, ad, bd, id, accf);
                            else tc::mma_bf16(dt, ad, bd, id, accf);
                        }
                    }
                }
                tc::mma_commit(&bars[buf]);
                last_commit = gt;
            }
        }
        tc::cp_async_wait<0>();   // no copy of this item outstanding (an early exit leaves some)
        if (p0 > 0) {   // sum_i (Re a_{i,0,q} - shift_q) into the float64 sums
#pragma unroll
            for (int u = 0; u < COV_PF; ++u) {
                const int it = threadIdx.x + COV_NT * u;
                if (it >= nslots) break;
                const int pr = it >> 5, q = 8 * (pr & (QBP - 1)) + (it & 7);
                if (q < p0) atomicAdd(&S.sum0[q], (double)s0acc[u]);
            }
        }
        __syncthreads();
        // the last commit covers every MMA issued before it
        if (ntiles > 0 && threadIdx.x == 0 && *okflag) {
            if (!tc::mbar_wait(&bars[(gt - 1) & 1], (uint32_t)(((gt - 1) >> 1) & 1), wb)) {
                ffb_flag(status, FFB_ERR_TIMEOUT);
                atomicExch(okflag, 0);
            }
        }
        tc::fence_after_sync();
        __syncthreads();   // okflag is read below only after this barrier
        if (ntiles > 0 && *okflag) {
            // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows q); row q of
            // block k keeps columns [rk, rk + pk) of its own k.  The warp loads
            // the 16-column groups spanning its lanes' ranges, every fourth
            // group per column set w / 4
            const int q = 32 * (warp & 3) + lane;
            int kq = -1, rk = 0, pq = 0;
            if (q < rows) {
                for (int k = sb.x; k < sb.y; ++k) {
                    const int r = S.off[k] - row0, pk = S.pk[k];
                    if (q >= r && q < r + pk) {
                        kq = k;
                        rk = r;
                        pq = pk;
                        break;
                    }
                }
            }
            int lo = (kq >= 0) ? rk : 1 << 20, hi = (kq >= 0) ? rk + pq : 0;
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            const int used = min(COV_NACC, ntiles);
            double *blk = (kq >= 0) ? S.acc + S.cov_off[kq] : nullptr;
            for (int c16 = (lo & ~15) + 16 * (warp >> 2); c16 < hi; c16 += 64) {
                float sum[16];
                tc::tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c16, sum);
                for (int a = 1; a < used; ++a) {
                    float v[16];
                    tc::tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(a * 128 + c16), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) sum[i] += v[i];
                }
                if (kq >= 0) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = c16 + i;
                        if (c >= rk && c < rk + pq) atomicAdd(&blk[(size_t)(q - rk) * pq + (c - rk)], (double)sum[i]);
                    }
                }
            }
        }
        // accumulator reads complete before the next item's MMAs overwrite them
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    // after a timeout the per-item wait above is skipped: the newest commit
    // covers every MMA this CTA issued, and they all finish before TMEM is
    // released (full budget; on the normal path the phase is already done)
    if (threadIdx.x == 0 && last_commit >= 0)
        tc::mbar_wait(&bars[last_commit & 1], (uint32_t)((last_commit >> 1) & 1), TC_BUDGET);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512u);
}

// one CTA per SM, so the 512-column TMEM allocation never waits for another CTA
static size_t tc_cov_smem(int prec) {
    const bool tf = (prec == FFB_TF32 || prec == FFB_TF32X3);
    const size_t nchunk = tf ? 2 : 1;   // 128-byte K chunks per 32-image tile
    return 1024 + 2 * (size_t)2 * nchunk * 128 * 128 + (size_t)COV_RS * COV_NT * COV_PF * sizeof(float2) + 64;
}

bool ffb_tc_cov_supported(ffb_plan_t p) {
    if (p->precision == FFB_FP32) return false;
    if (p->pmax > 128) return false;   // a block's rows live in one M = 128 tile
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return tc_cov_smem(p->precision) <= (size_t)optin;
}

template <int KIND, int NP>
static int launch_tc_cov(const CovGroup &g, int grid, int *status, cudaStream_t s, long long wb) {
    const size_t smem = tc_cov_smem(KIND == 0 ? FFB_TF32 : FFB_BF16);
    static int attr = 0;
    if (attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_tc_cov<KIND, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    // accumulator a takes the tiles t = a mod COV_NACC of an item: chains of
    // at most 128 images
    for (int i = 0; i < g.S; ++i)
        if (g.st[i].per > 128 * COV_NACC) return FFB_ERR_ARG;
    k_tc_cov<KIND, NP><<<grid, COV_NT, smem, s>>>(g, status, wb);
    return ffb_check_cuda(cudaGetLastError());
}

int ffb_launch_cov_group_tc(int precision, const CovGroup &g, int grid, int *status, cudaStream_t s,
                            long long wb) {
    if (g.nitems <= 0) return FFB_OK;
    if (grid <= 0) grid = ffb_cov_grid_default(precision);
    if ((int64_t)grid > g.nitems) grid = (int)g.nitems;
    int e;
    switch (precision) {
        case FFB_TF32: e = launch_tc_cov<0, 1>(g, grid, status, s, wb); break;
        case FFB_TF32X3: e = launch_tc_cov<0, 2>(g, grid, status, s, wb); break;
        case FFB_BF16: e = launch_tc_cov<1, 1>(g, grid, status, s, wb); break;
        case FFB_BF16X3: e = launch_tc_cov<1, 2>(g, grid, status, s, wb); break;
        default: return FFB_ERR_ARG;
    }
    return e;
}

int ffb_launch_cov_tc(ffb_plan_t p, const float *d_coef, int64_t n, cudaStream_t s) {
    CovGroup g;          // copied into the launch's parameters
    g.S = 1;
    g.tile_imgs = COV_TI;
    ffb_cov_stack(p, d_coef, n, true, &g.st[0]);
    g.st[0].item0 = 0;
    g.nitems = (int64_t)g.st[0].nk * ((n + g.st[0].per - 1) / g.st[0].per);
    ProfScope ps(p, FFB_KC_COV, s);
    const int e = ffb_launch_cov_group_tc(p->precision, g, 0, p->d_status, s, p->wait_budget);
    p->launches += 1;
    return e;
}
