// ffb_internal.cuh -- plan layout and device helpers shared by the CUDA
// translation units of the library (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/ffb.h"

#define FFB_MAX_RADIX_STAGES 16

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct FftPlanDev {
    int n;                          // transform length
    int nst;                        // number of Stockham stages
    int rad[FFB_MAX_RADIX_STAGES];  // radix of each stage (4, 2, 3, 5)
};

// kernel classes for the optional per-launch event timing (ffb_profile)
enum { FFB_KC_ROWS = 0, FFB_KC_COLS = 1, FFB_KC_INTERP = 2, FFB_KC_BESSEL = 3, FFB_KC_COV = 4,
       FFB_KC_COVAUX = 5, FFB_KC_EIG = 6, FFB_KC_ADJ_BESSEL = 7, FFB_KC_ADJ_RING = 8,
       FFB_KC_ADJ_COLS = 9, FFB_KC_ADJ_ROWS = 10, FFB_KC_FILTER = 11, FFB_KC_SETUP = 12,
       FFB_KC_GRID_INTERP = 13, FFB_KC_RING_FFT = 14, FFB_KC_ADJ_SPREAD = 15, FFB_NKC = 16 };

struct ProfEv {
    cudaEvent_t a, b;
    int cls;
};

// Default bound, in SM clock cycles, of every device-side wait of the
// tensor-core kernels (~2 s at 2 GHz); a wait that runs out latches
// FFB_ERR_TIMEOUT instead of spinning forever.
#define FFB_WAIT_BUDGET (4000000000LL)

#define FFB_HOST_SLOTS 3   // image parts in flight in ffb_expand_cov_host
struct ffb_plan_s {
    // problem
    int L, off;          // image size, pixel index offset (i = a - off)
    double c, R, eps;
    int precision;
    // basis
    int k_max, P, n_xi, n_theta, pmax;
    std::vector<int> p, offset;   // host, k_max+1
    std::vector<int> cov_off;     // host, k_max+2: offsets of blocks in packed C
    int cov_total;                // sum p_k^2
    // NUFFT
    int N, w, h, Mh;     // fine grid size, kernel width, halo, rows of the half grid
    double beta;         // ES kernel shape
    FftPlanDev fftN, fftT;
    int chunk;           // images per internal chunk
    int nq0;             // half-ring angles with cos(theta) >= 0 (fused path split)
    int fused;           // 1: grid held in shared memory (ffb_grid.cu); 2: as 1, in CTA-pair clusters
    // device tables (float64 setup results)
    double *d_zeros = nullptr;   // [P]
    double *d_xi = nullptr;      // [n_xi]
    double *d_wq = nullptr;      // [n_xi]
    double *d_B64 = nullptr;     // [P][n_xi]
    // device tables used by the hot path
    float *d_Bf = nullptr;       // [P][n_xi]   fp32 copy of B
    int *d_p = nullptr;          // [k_max+1]
    int *d_off = nullptr;        // [k_max+1]
    int *d_cov_off = nullptr;    // [k_max+2]
    float *d_corr = nullptr;     // [L] 1/Psi((a-off)/N)
    float2 *d_twN = nullptr;     // [N] e^{-2 pi i e/N}
    float2 *d_twT = nullptr;     // [n_theta]
    float2 *d_rad = nullptr;     // [n_xi] N xi_j as (hi, lo)
    float4 *d_ang = nullptr;     // [n_theta/2] (cos hi, cos lo, sin hi, sin lo)
    int4 *d_cov_work = nullptr;  // covariance work items (k, q0, q0', 0)
    int n_cov_work = 0;
    int4 *d_cov_sb = nullptr;    // tensor-core covariance super-blocks (k0, k1, first index, rows)
    int n_cov_sb = 0;
    // scratch (chunk-sized)
    float2 *d_H = nullptr;       // [chunk][N/2+1][L]
    float2 *d_G = nullptr;       // [chunk][Mh][N]
    float *d_Fhat = nullptr;     // [k_max+1][chunk][2][n_xi]
    float2 *d_Fpol = nullptr;    // [chunk][n_xi][n_theta/2] (fused path)
    float4 *d_nodes = nullptr;   // [blocks][9][units] phase-3 unit records (fused path)
    int2 *d_node_blk = nullptr;  // [blocks] (first node, node count), half 0 then half 1
    float4 *d_tunits = nullptr;  // separate-kernel path: tile unit records [blocks][19][256] (ffb_tile.cu)
    int4 *d_tblk = nullptr;      // [blocks] (first G row, first unwrapped column, first node, count)
    int *d_tnodes = nullptr;     // node lists of the tile blocks (t = j n_theta/2 + l)
    int ntblk = 0;               // tile blocks (0: the per-node interpolation kernel)
    int ring_direct = 0;         // 1: the register ring FFT (ffb_ring.cu) writes the quadrature
                                 //    operands from the polar buffer (fused path, and tiled plans
                                 //    with n_theta in {64, ..., 1024})
    float2 *d_twA = nullptr;     // [n_theta/32][32] ring FFT twiddles W^{j k1} (fused path)
    float2 *d_twG = nullptr;     // [N/32][32] grid FFT twiddles W_N^{j k1} (fused path)
    int node_nblk[2] = {0, 0};   // blocks per half
    // covariance state
    double *d_acc = nullptr;     // [cov_total] sum Re(a a^*), k = 0 shifted
    double *d_sum0 = nullptr;    // [p0] sum (a0 - shift)
    float *d_shift = nullptr;    // [p0]
    int64_t n_acc = 0;
    int shift_set = 0;
    // eig results
    double *d_Cfin = nullptr;    // [cov_total]
    double *d_mean = nullptr;    // [p0]
    double *d_evals = nullptr;   // [P]
    double *d_evecs = nullptr;   // [cov_total]
    double *d_eig_work = nullptr;  // Jacobi workspace of large blocks (V, and A above 166 rows)
    // denoising
    float2 *d_coef_den = nullptr;  // [den_cap][P]
    int64_t den_cap = 0;
    double *d_gain = nullptr;      // [P]
    float *d_M = nullptr;          // [cov_total] U diag(h) U^T per block
    int selected = 0;              // filter matrices valid
    int eig_ready = 0;             // d_evals / d_evecs hold eigenpairs
    // host-buffer entry point (ffb_expand_cov_host): a ring of FFB_HOST_SLOTS
    // device image buffers of host_cap images each, the coefficients of one
    // part, the copy stream and per-slot events (copy done, slot free again)
    float *d_hostimg = nullptr;
    float *d_hostcoef = nullptr;
    int64_t host_cap = 0;
    cudaStream_t h2d = nullptr;
    cudaEvent_t ev_copied[FFB_HOST_SLOTS] = {}, ev_free[FFB_HOST_SLOTS] = {};
    // status word written by kernels (first nonzero error wins)
    int *d_status = nullptr;
    // clock-cycle budget of the waits between the pipeline roles of the
    // tensor-core kernels (ffb_set_wait_budget); the drains of copies and
    // MMAs already issued always keep FFB_WAIT_BUDGET
    long long wait_budget = FFB_WAIT_BUDGET;
    int device = -1;     // the CUDA device the plan's tables live on
    int64_t launches = 0;
    // tensor-core operand tables and TMA descriptors (ffb_tc.cu)
    void *tc = nullptr;
    // optional per-launch timing
    int prof_on = 0;                 // 0 off, else the sampling stride
    size_t prof_used = 0;
    std::vector<ProfEv> prof;
    int64_t prof_calls[16] = {};     // launches per class since profiling was enabled
};

// FFB_OK when `p` is a plan and the current device is the one it was built
// on (its tables, scratch and the kernels' per-device state belong there);
// FFB_ERR_ARG otherwise.
int ffb_plan_here(ffb_plan_t p);
#define FFB_PLAN_HERE(p)                      \
    do {                                      \
        const int _here = ffb_plan_here(p);   \
        if (_here != FFB_OK) return _here;    \
    } while (0)

// Brackets one launch with events when profiling is on (host side).
struct ProfScope {
    ffb_plan_s *p;
    cudaStream_t s;
    int idx;
    ProfScope(ffb_plan_s *p_, int cls, cudaStream_t s_) : p(p_), s(s_), idx(-1) {
        if (!p->prof_on) return;
        // every prof_on-th launch of each class is timed (the first included)
        if (p->prof_calls[cls & 15]++ % p->prof_on != 0) return;
        if (p->prof_used == p->prof.size()) {
            ProfEv e;
            if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return;
            p->prof.push_back(e);
        }
        idx = (int)p->prof_used++;
        p->prof[idx].cls = cls;
        cudaEventRecord(p->prof[idx].a, s);
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecord(p->prof[idx].b, s);
    }
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ffb_flag(int *status, int code) {
    atomicCAS(status, 0, code);
}

// Programmatic dependent launch: a kernel launched with the
// programmatic-serialization attribute may start while the previous kernel
// in its stream runs; pdl_wait() returns once that kernel has completed and
// its memory operations are visible (immediately without the attribute);
// pdl_trigger() lets this kernel's own dependents launch once every CTA of it
// has executed it or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// L2 eviction-priority policies for data read once (evict first) and for
// data a later kernel of the step reads again (evict last), and accesses
// that carry them
// (no side effects: not volatile, so that the compiler hoists them out of loops)
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ldg_hint(const float *a, unsigned long long pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ldg_hint(const float2 *a, unsigned long long pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(void *a, unsigned v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(void *a, unsigned short v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(a), "h"(v), "l"(pol) : "memory");
}

// the launch attribute for it
static inline cudaLaunchAttribute ffb_pdl_attr() {
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
    return a;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs: V[m] = sum_r v[r] e^{-+2 pi i r m / R}.
template <bool INV>
__device__ __forceinline__ void dft2(float2 *v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <bool INV>
__device__ __forceinline__ void dft4(float2 *v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}
template <bool INV>
__device__ __forceinline__ void dft3(float2 *v) {
    const float s = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 t = cadd(v[1], v[2]);
    float2 u = csub(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 r = mul_mi<INV>(cscale(u, s));   // -i s u (forward)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}
template <bool INV>
__device__ __forceinline__ void dft5(float2 *v) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi/5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi/5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi/5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi/5)
    float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    float2 x0 = v[0];
    float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
    float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
    float2 q1 = mul_mi<INV>(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    float2 q2 = mul_mi<INV>(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
}

// One Stockham autosort pass sequence (decimation in time) executed by a
// group of `nthr` threads (thread index `t` within the group) on a length-n
// sequence in shared memory.  a: input, b: scratch; returns the buffer
// holding the result.  The caller synchronises the group between passes via
// `sync` (a functor) -- for a single warp this is __syncwarp().
// Stage s with radix R and Ns = product of earlier radices maps butterfly j
// (0 <= j < n/R) from a[j + r n/R] (twiddled by W_n^{r (j mod Ns) n/(Ns R)})
// to b[(j/Ns) Ns R + (j mod Ns) + r Ns].
template <bool INV, class Sync>
__device__ __forceinline__ float2 *smem_fft(float2 *a, float2 *b, const FftPlanDev &fp,
                                            const float2 *__restrict__ tw, int t, int nthr,
                                            Sync sync) {
    const int n = fp.n;
    int Ns = 1;
    for (int s = 0; s < fp.nst; ++s) {
        const int R = fp.rad[s];
        const int nb = n / R;
        const int tstep = n / (Ns * R);
        for (int j = t; j < nb; j += nthr) {
            const int k = j % Ns;
            float2 v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) v[r] = a[j + r * nb];
#pragma unroll
            for (int r = 1; r < 5; ++r) {
                if (r < R) {
                    int e = (r * k * tstep) % n;
                    float2 wv = __ldg(&tw[e]);
                    if (INV) wv.y = -wv.y;
                    v[r] = cmul(v[r], wv);
                }
            }
            if (R == 4) dft4<INV>(v);
            else if (R == 2) dft2<INV>(v);
            else if (R == 3) dft3<INV>(v);
            else dft5<INV>(v);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) b[base + r * Ns] = v[r];
        }
        sync();
        float2 *tmp = a;
        a = b;
        b = tmp;
        Ns *= R;
    }
    return a;
}

struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// float32 rounded to the nearest tf32 (10 explicit mantissa bits), ties away
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    return __uint_as_float(u);
}

// Operand formats the ring FFT can write for the radial quadrature.
enum { FFB_FMT_F32 = 0, FFB_FMT_TF32 = 1, FFB_FMT_TF32X2 = 2, FFB_FMT_BF16 = 3, FFB_FMT_BF16X2 = 4 };

// Exponential-of-semicircle kernel psi(x) = exp(beta (sqrt(1 - z^2) - 1)),
// z = 2x/w, |x| < w/2, in fine-grid units, evaluated as
// exp(-beta z^2 / (1 + sqrt(1 - z^2))): the exponent carries a small relative
// error instead of the absolute error of sqrt(u) - 1 near the centre, so the
// approximate square root and quotient suffice (weight error <= ~2e-7).
__device__ __forceinline__ float es_kernel(float x, float two_over_w, float beta) {
    const float z = x * two_over_w;
    const float z2 = z * z;
    const float u = 1.0f - z2;
    if (!(u > 0.0f)) return 0.0f;
    return __expf(-__fdividef(beta * z2, 1.0f + u * rsqrtf(u)));
}

// J_k(x), x >= 0, by Miller's backward recurrence: starting far above both k
// and x with (t_{M+1}, t_M) = (0, tiny), t_{m-1} = (2m/x) t_m - t_{m+1} is
// proportional to J_{m-1}(x) (the minimal solution); the constant follows from
// J_0 + 2 sum_{m>=1} J_{2m} = 1.  Values are rescaled when they grow large.
__device__ __forceinline__ double bessel_j_miller(int k, double x) {
    if (x <= 0.0) return (k == 0) ? 1.0 : 0.0;
    double top = fmax((double)k, x);
    int M = (int)(top + 16.0 * cbrt(0.5 * top) + 24.0);
    M += (M & 1);  // even start
    double tp1 = 0.0, t = 1e-300, sum = 0.0, jk = 0.0;
    for (int m = M; m >= 1; --m) {
        // here t = t_m, tp1 = t_{m+1}
        if (m == k) jk = t;
        if ((m & 1) == 0) sum += 2.0 * t;
        double tm1 = (2.0 * m / x) * t - tp1;
        tp1 = t;
        t = tm1;
        if (fabs(t) > 1e250) {
            t *= 1e-250;
            tp1 *= 1e-250;
            sum *= 1e-250;
            jk *= 1e-250;
        }
    }
    // t = t_0
    if (k == 0) jk = t;
    sum += t;
    return jk / sum;
}

// Host helpers (implemented in ffb_plan.cu).
int ffb_check_cuda(cudaError_t e);
int ffb_ensure_scratch(ffb_plan_t plan);
int ffb_ensure_scratch_grid(ffb_plan_t plan);
// true when two buffers of rb rings of n_theta complex values each fit in
// the shared memory one CTA may opt in to (the ring DFT kernels' staging)
bool ffb_ring_buffers_fit(int n_theta, int rb);
bool ffb_fused_supported(ffb_plan_t plan);
int ffb_fused_prepare(ffb_plan_t plan, cudaStream_t s);
int ffb_fused_mode(ffb_plan_t plan);   // 1 plain, 2 cluster variant of the fused kernel
int ffb_ring_prepare(ffb_plan_t plan, cudaStream_t s);   // ring FFT twiddle table (fused path)
// adjoint spreading of m images' half-ring values (polar-buffer layout) into
// the zeroed extended grid [m][Mh][N] with the fused path's unit table
int ffb_launch_fused_spread(ffb_plan_t plan, const float2 *Gpol, int m, float2 *Gext, cudaStream_t s);
// n_after: images that follow the chunk [i0, i0 + m) in d_images (the
// kernel prefetches one wave ahead into L2, never past them)
// planes: write the polar samples as the bf16 hi / lo planes of the
// tensor-core ring DFT (into the plan's polar buffer) instead of float32
int ffb_launch_fused_polar(ffb_plan_t plan, const float *d_images, int64_t i0, int m, float2 *Fpol,
                           cudaStream_t s, bool pdl = false, int64_t n_after = 0, bool planes = false);
struct RingOut {
    int fmt;           // FFB_FMT_*
    void *p0, *p1;     // planes (FFB_FMT_F32: p0 = float32 spectra), at the launch's first image
    int ld;            // row length of the planes (>= n_xi)
    int lead;          // images per k in the planes
};
int ffb_launch_ring_fft(ffb_plan_t plan, int m, const float2 *Fpol, const RingOut &out, cudaStream_t s);
int ffb_launch_ring_ifft(ffb_plan_t plan, int m, const float *Yhat, float2 *Gpol, cudaStream_t s);
int ffb_tc_prepare(ffb_plan_t plan, cudaStream_t s, RingOut *out);
// ring DFT on the tensor cores (ffb_tc.cu): whether the plan takes it, and
// one chunk's launch from the bf16 polar planes into the operand planes
bool ffb_tc_dft_ok(ffb_plan_t plan);
int ffb_launch_tc_dft(ffb_plan_t plan, int m, const RingOut &out, cudaStream_t s);
// chunks whose ring spectra one tensor-core quadrature launch takes (>= 1;
// valid after ffb_tc_prepare)
int ffb_tc_group(ffb_plan_t plan);
// grouped tensor-core quadrature over several plans (ffb_tc.cu): descriptor
// size, the plan's padded block width, one stack's descriptor (host memory),
// the launch shapes to tune over, the launch
size_t ffb_tc_stack_bytes();
int ffb_tc_bn(ffb_plan_t plan);
int ffb_tc_stack_fill(ffb_plan_t plan, float *coef, int nimg, int item0, void *dst, int *nitems);
int ffb_tc_group_shapes(int precision, int BNmax, int *per_sm, int *nst);
int ffb_tc_group_bessel(int precision, const void *d_stacks, int S, int nitems, int BNmax, int per_sm, int nst,
                        int *status, long long wait_budget, cudaStream_t s);
int ffb_tc_split_planes(ffb_plan_t plan, cudaStream_t s);
// a1-a4 of images [g0, g1) (one group of chunks) into the plan's quadrature
// operands, without the quadrature (ffb_api.cu)
int ffb_expand_part(ffb_plan_t plan, const float *d_images, int64_t g0, int64_t g1, cudaStream_t s);
// tiled interpolation of the separate-kernel path (ffb_tile.cu)
int ffb_tile_prepare(ffb_plan_t plan, cudaStream_t s);
int ffb_launch_tile_polar(ffb_plan_t plan, int nimg, float2 *F, cudaStream_t s);
int ffb_launch_tile_spread(ffb_plan_t plan, int nimg, const float2 *Gpol, float2 *Gext, cudaStream_t s);

// Launchers implemented in ffb_nufft.cu / ffb_gemm.cu / ffb_eig.cu.
int ffb_launch_grid(ffb_plan_t plan, const float *d_images, int64_t i0, int nimg, cudaStream_t s);
int ffb_launch_polar(ffb_plan_t plan, int nimg, float *d_F, cudaStream_t s);
int ffb_launch_interp_ring(ffb_plan_t plan, int nimg, cudaStream_t s);
int ffb_launch_bessel(ffb_plan_t plan, int nimg, float *d_coef_chunk, bool planes_ready, cudaStream_t s);
int ffb_launch_bessel_tc(ffb_plan_t plan, int nimg, float *d_coef_chunk, bool planes_ready, cudaStream_t s);
bool ffb_tc_supported(ffb_plan_t plan);
bool ffb_tc_cov_supported(ffb_plan_t plan);
int ffb_launch_cov_tc(ffb_plan_t plan, const float *d_coef, int64_t n, cudaStream_t s);
void ffb_tc_release(ffb_plan_t plan);
int ffb_launch_cov(ffb_plan_t plan, const float *d_coef, int64_t n, cudaStream_t s);
int ffb_launch_cov_shift(ffb_plan_t plan, const float *d_coef, int64_t n, cudaStream_t s);
int ffb_launch_cov_final(ffb_plan_t plan, cudaStream_t s);
int ffb_launch_eig(ffb_plan_t plan, cudaStream_t s);

// ---- covariance over one or several stacks in one launch (a6/a7) ----------
// A launch covers the stacks st[0..S); stack s contributes items
// [item0, item0 + nk * ceil(n / per)): item i of the stack is image range
// i / nk (per images) of block or tile i % nk.  The table travels as a kernel
// parameter (about 6 KB for 64 stacks), so a captured graph keeps its own copy.
#define FFB_GROUP_MAX 64
struct CovStack {
    const float2 *coef;     // [n][P] coefficients of the stack
    int64_t n;              // images
    int64_t item0;          // first item of the stack in the launch
    const int *pk, *off, *cov_off;
    const int4 *work;       // FP32 kernel: (k, q0, q1) tiles; tensor cores: super-blocks
    const float *shift;     // k = 0 pilot mean
    double *acc, *sum0;     // float64 accumulators
    int P;
    int nk;                 // items per image range: super-blocks (tensor cores) or tiles (FP32)
    int per;                // images per item
    int pmax;
};
struct CovGroup {
    int S;
    int tile_imgs;          // tensor cores: images per MMA tile (32)
    int64_t nitems;
    CovStack st[FFB_GROUP_MAX];
};
__device__ __forceinline__ int cov_stack_of(const CovGroup &g, int64_t item) {
    int s = 0;
    while (s + 1 < g.S && g.st[s + 1].item0 <= item) ++s;
    return s;
}
// fills st for plan p (item0 and per are set by the caller); tc selects the
// item kind: k blocks (tensor cores) or the plan's FP32 tile list
void ffb_cov_stack(ffb_plan_t p, const float *d_coef, int64_t n, bool tc, CovStack *st);
// covariance launches over a stack table; precision selects the kernel
// (FFB_FP32: float32 tiles; otherwise the tensor-core form); grid <= 0 picks
// one CTA per SM (tensor cores) or a full wave (FP32)
int ffb_launch_cov_group(int precision, const CovGroup &g, int grid, int *status, cudaStream_t s);
int ffb_cov_grid_default(int precision);
int ffb_launch_cov_group_tc(int precision, const CovGroup &g, int grid, int *status, cudaStream_t s,
                            long long wait_budget = FFB_WAIT_BUDGET);
int ffb_expand_on(ffb_plan_t plan, const float *d_images, int64_t n, float *d_coef, cudaStream_t s);
int ffb_launch_adjoint(ffb_plan_t plan, const float *d_coef, int64_t n, float *d_images,
                       cudaStream_t s);
int ffb_launch_filter_matrix(ffb_plan_t plan, cudaStream_t s);
int ffb_launch_filter(ffb_plan_t plan, const float *d_coef_in, int64_t n, float *d_coef_out, int flags,
                      cudaStream_t s);
int ffb_launch_weight(ffb_plan_t plan, const float *d_coef_in, int64_t n, float *d_coef_out, cudaStream_t s);
