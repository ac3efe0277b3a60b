// ffb_grid.cu -- steps a1-a3 with the oversampled grid held in shared memory
// (the type-2 NUFFT of Eq. nufft onto the polar nodes of Sec. III).
//
// One CTA per (image, half).  Half 0 owns the polar nodes with xi1 >= 0
// (theta in [0, pi/2]), half 1 those with xi1 < 0 (theta in (pi/2, pi)); all
// have xi2 >= 0.  The grid values a half needs are G[m1][m2] for
// m2 in [-h, N/2 + h] and m1 in [-h, N/2 + h] (half 0) or [-N/2 - h, h]
// (half 1): a (N/2 + 1 + 2h)^2 block that fits in one SM's shared memory
// for N <= 256 (137 x 137 complex = 150 KB at N = 256, w = 8).
//
// Phase 1  rows: for pixel rows a1 (two per complex FFT, one FFT per half
//          warp at N = 256, per warp at N = 128), the length-N DFT
//          over i2 of I(i) corr(i1) corr(i2) placed at i2 mod N; the outputs
//          m2 in [-h, N/2 + h] are stored in column a1 of S[m2 + h][.].
// Phase 2  columns: for each m2 row of S, the length-N DFT over i1 (entries
//          placed at i1 mod N); the half's m1 range overwrites the row in
//          place (the row is read completely before it is written).
// Phase 3  interpolation of the half's nodes from S (w x w taps of the ES
//          kernel with weights from the plan), the result written to the
//          polar buffer F[img][j][l], l < n_theta/2 (float32 pairs, or the
//          bf16 hi / lo planes of u and v for the tensor-core ring DFT).
// The ring DFT of Eq. 1DFFT then completes every half ring with
// F(theta + pi) = conj F(theta): the register FFT of ffb_ring.cu, or, for the
// BF16x3 plans at n_theta = 512, the tensor-core contraction of ffb_tc.cu.
//
// Phases 1 and 2 are the same for both halves.  Where clusters of two CTAs
// fill the GPU, the two CTAs of an image form one and split them: each
// transforms half of the pixel-row pairs and half of the S rows, and sends
// the peer what it needs through distributed shared memory (contiguous row
// segments after phase 1, the peer's column range of every row it
// transformed in phase 2).
//
// Node order in phase 3.  A node gathers the W x W window of S at
// S[r0][c0] (W = 8).  Up to four nodes whose window origins lie in one 2 x 2
// box (r0 or r0 + 1, c0 or c0 + 1) form a unit: one thread reads the 9 x 9
// union of their windows once and forms all their results, 81 gathers for
// about 3.4 nodes instead of 64 per node (phase 3 is bound by the
// shared-memory pipe).  One 8-byte load of a half warp takes a single
// wavefront when the 16 union origins r0 * SLD + c0 fall in distinct 8-byte
// bank slots (the origin mod 16), so the units are ordered into half warps
// with distinct slots; a unit whose nodes all sit in the union's first
// column (row) may start its union one column (row) earlier, which the plan
// uses to even out the slots' unit counts.  Everything here depends on the
// geometry alone and is built by the plan in float64 (ffb_fused_prepare):
// blocks of consecutive nodes t = j nl + l, at most one unit per thread, and
// per unit the origin, the node slots and every node's weights over the
// union's 9 columns and 9 rows (zero outside its own window; 304 bytes per
// unit, about 3 MB at N = 256, read from L2 by every CTA).  The kernel
// stages a block's results in shared memory and stores them in natural
// order.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ffb_fft.cuh"

// 24 warps: 80 registers per thread hold a four-node unit's 36 column
// weights and accumulators without spills (at 32 warps, 64 registers, they
// spill; measured slower)
#define FUS_WARPS 24                 // warps per CTA, each with an N-entry FFT buffer
#define FUS_NT (32 * FUS_WARPS)      // threads per CTA
#define FUS_GU FUS_NT  // units per phase-3 block (at most; one per thread)
#define FUS_NU 4       // nodes per unit (at most)
#define FUS_UW 9       // union side: W + 1
#define FUS_REC 19     // float4 planes of a unit record: 9 column, 9 row, 1 meta

// rows and columns of the shared-memory grid block: MH (odd) rows and
// columns hold the half plane; one more zero row and two more zero columns
// let a unit's 9 x 9 union start at the last window origin (its extra row or
// column then carries zero weights); the row pitch SLD stays odd
__host__ __device__ constexpr int fus_mh(int N, int W) { return N / 2 + 1 + 2 * ((W + 1) / 2); }
__host__ __device__ constexpr int fus_sld(int N, int W) { return fus_mh(N, W) + 2; }
__host__ __device__ constexpr int fus_rows(int N, int W) { return fus_mh(N, W) + 1; }

// ---------------------------------------------------------------------------
// Length-N forward DFT of a sequence whose only nonzeros are the L = N/2
// values placed at (a - L/2) mod N, a = lane + 32 q, given in z[q] (N = 128,
// 256), by one warp as a four-step FFT.  With N = 32 M, index l = 32 m + j
// (lane j) and k = k1 + M k2:
//   X_k = sum_j W^{j k1} [sum_m s_{32m+j} W_M^{m k1}] W_32^{j k2},  W = e^{-2 pi i/N}.
// The nonzeros sit at m in {0, 1, M-2, M-1} (N = 256) or {0, M-1} (N = 128),
// so the length-M DFT over m starts from two half-zero length-4 DFTs
// (a + d i^k for inputs (a, 0, 0, d)).  After the twiddle W^{j k1}, one
// transpose through the warp's buffer (row k1, column rotated by k1 R,
// R = 32/M: conflict-free) gives lane (g = k1, r) the values j = r + R i;
// a length-M DFT over i, the twiddle W_32^{r k2'} and a length-R DFT across
// the group's lanes (radix-2 decimation in frequency by XOR shuffles, lane r
// ends with t = bitreverse(r)) give X_k, k = g + M (k2' + M t).  X is left in
// the buffer in natural order at position fswz<N>(k): the XOR with the bits
// above M^2 spreads the lanes of one write over 16 bank slots, and runs of
// consecutive k stay contiguous for the readers.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ int fswz(int k) {
    return (N == 256) ? (k ^ ((k >> 6) << 2)) : (k ^ ((k >> 4) << 1));
}

template <int N>
__device__ __forceinline__ void warp_fft_halfzero(const float2 *z, float2 *buf, const float2 *__restrict__ tw,
                                                  const float2 *__restrict__ twA, int lane) {
    static_assert(N == 128 || N == 256, "N in {128, 256}");
    constexpr int M = N / 32, R = 32 / M;
    float2 x[M];
    if constexpr (N == 256) {
        // z[2], z[3] at m = 0, 1; z[0], z[1] at m = 6, 7: even-m DFT4 of
        // (z2, 0, 0, z0) in x[0..3], odd-m DFT4 of (z3, 0, 0, z1) in x[4..7]
        {
            const float2 a = z[2], d = z[0];
            x[0] = cadd(a, d); x[1] = make_float2(a.x - d.y, a.y + d.x);
            x[2] = csub(a, d); x[3] = make_float2(a.x + d.y, a.y - d.x);
        }
        {
            const float2 b = z[3], e = z[1];
            x[4] = cadd(b, e); x[5] = make_float2(b.x - e.y, b.y + e.x);
            x[6] = csub(b, e); x[7] = make_float2(b.x + e.y, b.y - e.x);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // radix-2 combination with W8^k
            float2 t = x[k + 4];
            if (k == 1) t = make_float2(FFB_R2 * (t.x + t.y), FFB_R2 * (t.y - t.x));
            if (k == 2) t = make_float2(t.y, -t.x);
            if (k == 3) t = make_float2(FFB_R2 * (t.y - t.x), -FFB_R2 * (t.x + t.y));
            const float2 e0 = x[k];
            x[k] = cadd(e0, t);
            x[k + 4] = csub(e0, t);
        }
    } else {
        // z[1] at m = 0, z[0] at m = 3
        const float2 a = z[1], d = z[0];
        x[0] = cadd(a, d); x[1] = make_float2(a.x - d.y, a.y + d.x);
        x[2] = csub(a, d); x[3] = make_float2(a.x + d.y, a.y - d.x);
    }
    // W^{lane k1} from the plan's table [k1][lane] (coalesced)
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) x[k1] = cmul(x[k1], __ldg(&twA[k1 * 32 + lane]));
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) buf[k1 * 32 + ((lane + k1 * R) & 31)] = x[k1];
    __syncwarp();
    const int g = lane / R, r = lane % R;
#pragma unroll
    for (int i = 0; i < M; ++i) x[i] = buf[g * 32 + ((r + R * i + g * R) & 31)];
    __syncwarp();
    dft_reg<M>(x);
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) x[k2] = cmul(x[k2], __ldg(&tw[(r * k2 * (N / 32)) & (N - 1)]));
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
        const bool up = (r & h) != 0;
        // the last stage (h = 1) has the twiddle W^0 = 1
        const float2 w = (h > 1) ? __ldg(&tw[(r & (h - 1)) * (N / (2 * h))]) : make_float2(1.f, 0.f);
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            const float2 pv = make_float2(__shfl_xor_sync(0xffffffffu, x[k2].x, h),
                                          __shfl_xor_sync(0xffffffffu, x[k2].y, h));
            const float2 d = csub(pv, x[k2]);
            x[k2] = up ? ((h > 1) ? cmul(d, w) : d) : cadd(x[k2], pv);
        }
    }
    int t = 0;
    for (int b = 1; b < R; b <<= 1) t = (t << 1) | ((r & b) ? 1 : 0);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) buf[fswz<N>(g + M * (k2 + M * t))] = x[k2];
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Length-256 forward DFT of the same half-zero sequence (nonzeros at
// (a - 64) mod 256, a < 128) by 16 lanes, one half of a warp, as a 16 x 16
// four-step: index l = 16 m + j (lane j of the half), k = k1 + 16 k2,
//   X_k = sum_j W^{j k1} [sum_m s_{16m+j} W_16^{m k1}] W_16^{j k2},  W = e^{-2 pi i/256}.
// xin[t] holds s at m = t (t < 4) and m = 8 + t (t >= 4), the only nonzero
// m; the length-16 DFT over m therefore starts from four half-zero length-4
// DFTs.  After the twiddle W^{j k1} (plan table [k1][j]) one transpose
// through the half's 128-entry buffer, in two rounds of eight k1 each
// (position rotated by k1: conflict-free), gives lane j the values of k1 = j
// over all sixteen j; a length-16 DFT over them leaves X_{j + 16 k2} in
// y[k2].  No cross-lane shuffles: two transforms per warp, each with about
// 40 % fewer instructions than the whole-warp form above.  Phase 1 at
// N = 256 uses it (its 32 row pairs per CTA then take one round of the 24
// warps instead of two); in phase 2 the outputs' way back into the rows
// costs more than it saves, and phase 2 keeps the whole-warp form.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void half_fft256_halfzero(const float2 (&xin)[8], float2 (&y)[16], float2 *hbuf,
                                                     const float2 *__restrict__ twH, int j) {
    // pass A: m = 4 n1 + n2 with n1 in {0, 3}: DFT4 over n1 of (a, 0, 0, d)
    float2 u[4][4];   // u[n2][q] = that DFT4, times W_16^{n2 q}
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        const float2 a = xin[n2], d = xin[4 + n2];
        const float2 v[4] = {cadd(a, d), make_float2(a.x - d.y, a.y + d.x), csub(a, d),
                             make_float2(a.x + d.y, a.y - d.x)};
#pragma unroll
        for (int q = 0; q < 4; ++q) u[n2][q] = (n2 * q == 0) ? v[q] : cmul(v[q], w16(n2 * q));
    }
    float2 x[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 v[4] = {u[0][q], u[1][q], u[2][q], u[3][q]};
        dft4<false>(v);
#pragma unroll
        for (int p = 0; p < 4; ++p) x[q + 4 * p] = v[p];
    }
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) x[k1] = cmul(x[k1], __ldg(&twH[k1 * 16 + j]));
    // transpose, k1 < 8 then k1 >= 8: entry (k1 mod 8, j) at 16 (k1 mod 8) + ((j + k1) mod 16)
#pragma unroll
    for (int rnd = 0; rnd < 2; ++rnd) {
#pragma unroll
        for (int k1 = 8 * rnd; k1 < 8 * rnd + 8; ++k1) hbuf[(k1 - 8 * rnd) * 16 + ((j + k1) & 15)] = x[k1];
        __syncwarp();
        if ((j >> 3) == rnd) {
#pragma unroll
            for (int i = 0; i < 16; ++i) y[i] = hbuf[(j - 8 * rnd) * 16 + ((i + j) & 15)];
        }
        __syncwarp();
    }
    dft_reg<16>(y);
}

// distributed shared memory of a thread-block cluster: a float2 store into the
// peer CTA's shared memory (cluster-space address from mapa), and the
// cluster-wide barrier with release / acquire ordering of shared memory
__device__ __forceinline__ void st_peer(unsigned addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// CL: the two CTAs of an image form a cluster and split the row and column
// transforms, which are the same for both halves: each computes half of them
// and writes the results into its own and its peer's grid block.
template <int N, int W, bool CL>
__global__ void __launch_bounds__(FUS_NT, 1)
k_grid_interp_half(const float *__restrict__ images, int off, const float *__restrict__ corr,
                   const float2 *__restrict__ tw, const float2 *__restrict__ twA, int n_xi, int n_theta, int nq0,
                   const float4 *__restrict__ units, const int2 *__restrict__ blocks, int nblk0, int nblk1,
                   float2 *__restrict__ Fpol, int *status, int wave, int n_after,
                   __nv_bfloat16 *__restrict__ planes, long long pstride) {
    constexpr int L = N / 2;
    constexpr int H = (W + 1) / 2;
    constexpr int MH = fus_mh(N, W);              // rows of S (m2 + h)
    constexpr int SLD = fus_sld(N, W);            // row length of S
    constexpr int GN = FUS_WARPS * N / 2;         // nodes per block at most (two staged blocks)
    constexpr int SR = fus_rows(N, W);            // rows of S including the zero row
    extern __shared__ float2 smz[];
    float2 *S = smz;                               // [SR][SLD]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *buf = smz + SR * SLD + warp * N;   // this warp's FFT buffer
    const int half = blockIdx.x;
    const int img = blockIdx.y;
    const float *im = images + (size_t)img * L * L;
    pdl_trigger();
    // L2 prefetches (hints, with no completion to wait for), one bulk copy of
    // half `half` of an image's pixel rows each: this image's, so that the
    // transform rounds after the first find them in L2, and the image that
    // the CTA one wave later reads (img + wave of this launch, else of the
    // images that follow it), so that its first round does too
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(L / 2 * L * 4);
        const float *own = images + ((size_t)img * L + (size_t)half * (L / 2)) * L;
        if ((reinterpret_cast<uintptr_t>(own) & 15) == 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(own)), "r"(bytes)
                         : "memory");
        const int tgt = img + wave;
        if (wave > 0 && tgt < (int)gridDim.y + n_after) {
            const float *nxt = images + ((size_t)tgt * L + (size_t)half * (L / 2)) * L;
            if ((reinterpret_cast<uintptr_t>(nxt) & 15) == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(nxt)),
                             "r"(bytes)
                             : "memory");
        }
    }
    // the zero row below the half plane (no transform writes it)
    for (int i = threadIdx.x; i < SLD; i += FUS_NT) S[MH * SLD + i] = make_float2(0.f, 0.f);
    // cluster: the peer's S in the cluster window, this CTA's share of the
    // transforms (every second one)
    unsigned peerS = 0;
    int part = 0, nparts = 1;
    if constexpr (CL) {
        unsigned rank;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
        const unsigned own = (unsigned)__cvta_generic_to_shared(smz);
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(peerS) : "r"(own), "r"(rank ^ 1u));
        part = (int)rank;
        nparts = 2;
    }

    // ---- phase 1: row transforms (two pixel rows per complex FFT) --------
    // (cluster: this CTA's pixel rows are a1 in [part L/2, (part + 1) L/2))
    bool bad = false;
    // N = 256: one row pair per half warp (half_fft256_halfzero); half hw of
    // the warp takes pair slot 2 warp + hw, both halves run every step
    const int hw = lane >> 4, j16 = lane & 15;
    float2 *hbuf = buf + hw * (N / 2);
    const float2 *twH = twA + N;      // W^{j k1}, [16][16], after the warp FFT's table
    if constexpr (N == 256) {
        static_assert(N != 256 || (L == 128 && H == 4 && MH == 137), "half-warp FFT layout");
        const int nrp = L / 2 / nparts;
        for (int q0 = 2 * warp; q0 < nrp; q0 += 2 * FUS_WARPS) {
            const int q = q0 + hw;
            const bool act = q < nrp;
            const int a1 = 2 * (part * nrp + (act ? q : 0));
            const float c1 = corr[a1], c2 = corr[a1 + 1];
            float2 xin[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int a2 = (t < 4) ? (L / 2 + 16 * t + j16) : (16 * (t - 4) + j16);
                float xv = 0.f, yv = 0.f;
                if (act) {
                    // pixels are read once: evict first (the unit table and
                    // the polar buffer then keep their L2 lines)
                    const unsigned long long pf = l2_evict_first();
                    xv = ldg_hint(&im[(size_t)a1 * L + a2], pf);
                    yv = ldg_hint(&im[(size_t)(a1 + 1) * L + a2], pf);
                }
                bad |= !(isfinite(xv) && isfinite(yv));
                const float ca = corr[a2];
                xin[t] = make_float2(xv * c1 * ca, yv * c2 * ca);
            }
            float2 Z[16];
            half_fft256_halfzero(xin, Z, hbuf, twH, j16);
            // the two real rows' spectra from Z_m and conj Z_{N-m}, through the
            // half's buffer in two rounds: k in [0, 64) u [192, 256) (pairs of
            // m in [0, 64) u [252, 256): rows e in [0, 68)), then k in
            // [64, 192) (m in [65, 132]: e in [69, 136]); slot k2 of lane j16
            // is k = j16 + 16 k2.  Row e = 68 (m = 64, partner 192) straddles
            // the rounds: lane 0 holds both (k2 = 4, 12) and writes it.
            if (act && j16 == 0) {
                const float2 Zm = Z[4], Zc = cconj(Z[12]);
                const float2 D = csub(Zm, Zc);
                S[68 * SLD + a1] = make_float2(0.5f * (Zm.x + Zc.x), 0.5f * (Zm.y + Zc.y));
                S[68 * SLD + a1 + 1] = make_float2(0.5f * D.y, -0.5f * D.x);
            }
#pragma unroll
            for (int rnd = 0; rnd < 2; ++rnd) {
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) {
                    const bool in0 = (k2 < 4 || k2 >= 12);
                    if (in0 == (rnd == 0)) {
                        const int k = j16 + 16 * k2;
                        hbuf[rnd == 0 ? (k < 64 ? k : k - 128) : k - 64] = Z[k2];
                    }
                }
                __syncwarp();
                const int e0 = (rnd == 0) ? 0 : 69, e1 = (rnd == 0) ? 68 : MH;
                for (int e = e0 + j16; e < e1; e += 16) {
                    const int m = (e - H) & (N - 1), mc = (N - m) & (N - 1);
                    const int pm = (rnd == 0) ? (m < 64 ? m : m - 128) : m - 64;
                    const int pc = (rnd == 0) ? (mc < 64 ? mc : mc - 128) : mc - 64;
                    const float2 Zm = hbuf[pm];
                    const float2 Zc = cconj(hbuf[pc]);
                    const float2 D = csub(Zm, Zc);
                    if (act) {
                        S[e * SLD + a1] = make_float2(0.5f * (Zm.x + Zc.x), 0.5f * (Zm.y + Zc.y));
                        S[e * SLD + a1 + 1] = make_float2(0.5f * D.y, -0.5f * D.x);
                    }
                }
                __syncwarp();
            }
        }
    } else {
        for (int rp = part * (L / 2 / nparts) + warp; rp < (part + 1) * (L / 2 / nparts); rp += FUS_WARPS) {
            const int a1 = 2 * rp;
            float x[L / 32], y[L / 32];
#pragma unroll
            for (int q = 0; q < L / 32; ++q) {
                x[q] = __ldg(&im[(size_t)a1 * L + lane + 32 * q]);
                y[q] = __ldg(&im[(size_t)(a1 + 1) * L + lane + 32 * q]);
            }
            const float c1 = corr[a1], c2 = corr[a1 + 1];
            float2 z[L / 32];
#pragma unroll
            for (int q = 0; q < L / 32; ++q) {
                const int a2 = lane + 32 * q;
                bad |= !(isfinite(x[q]) && isfinite(y[q]));
                const float ca = corr[a2];
                z[q] = make_float2(x[q] * c1 * ca, y[q] * c2 * ca);
            }
            warp_fft_halfzero<N>(z, buf, tw, twA, lane);
            for (int e = lane; e < MH; e += 32) {
                const int m = (e - H) & (N - 1);
                const float2 Z = buf[fswz<N>(m)];
                const float2 Zc = cconj(buf[fswz<N>((N - m) & (N - 1))]);
                const float2 D = csub(Z, Zc);
                S[e * SLD + a1] = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
                S[e * SLD + a1 + 1] = make_float2(0.5f * D.y, -0.5f * D.x);
            }
            __syncwarp();
        }
    }
    if (bad) ffb_flag(status, FFB_ERR_NONFINITE);
    __syncthreads();
    if constexpr (CL) {
        // the peer transforms the rows e = 1 - part (mod 2) of S: send it this
        // CTA's half of each, as contiguous row segments
        for (int e = (part ^ 1) + 2 * warp; e < MH; e += 2 * FUS_WARPS) {
            const int i0 = e * SLD + part * (L / 2);
            for (int a = lane; a < L / 2; a += 32) st_peer(peerS + 8u * (unsigned)(i0 + a), S[i0 + a]);
        }
        cluster_sync_all();
    }

    // ---- phase 2: column transforms, in place per row of S ---------------
    // (cluster: a row is transformed once and both halves' columns written)
    const int m1lo = (half == 0) ? -H : -(N / 2) - H;
    const int m1lo_peer = (half == 0) ? -(N / 2) - H : -H;
    for (int e = part + nparts * warp; e < MH; e += nparts * FUS_WARPS) {
        float2 *row = S + e * SLD;
        float2 z[L / 32];
#pragma unroll
        for (int q = 0; q < L / 32; ++q) z[q] = row[lane + 32 * q];
        warp_fft_halfzero<N>(z, buf, tw, twA, lane);
        for (int c = lane; c < MH; c += 32) row[c] = buf[fswz<N>((c + m1lo) & (N - 1))];
        if (lane < SLD - MH) row[MH + lane] = make_float2(0.f, 0.f);
        if constexpr (CL) {
            const unsigned prow = peerS + 8u * (unsigned)(e * SLD);
            for (int c = lane; c < MH; c += 32) st_peer(prow + 8u * c, buf[fswz<N>((c + m1lo_peer) & (N - 1))]);
            if (lane < SLD - MH) st_peer(prow + 8u * (MH + lane), make_float2(0.f, 0.f));
        }
        __syncwarp();
    }
    // (cluster: the peer's writes into this block are complete and visible,
    // and no CTA touches its peer's shared memory after this barrier)
    if constexpr (CL) cluster_sync_all();
    else __syncthreads();

    // the polar buffer may still be read by the previous kernel (the ring DFT
    // of the previous chunk) when this launch started early
    pdl_wait();

    // ---- phase 3: interpolation of this half's nodes -----------------------
    // block b of the half covers the nodes t in [t0, t0 + cnt); unit record s
    // holds, as FUS_REC planes of GU float4:
    //   plane q      (q < 9)  the column weights of union column q, one per
    //                         node slot: (wx_0[q], wx_1[q], wx_2[q], wx_3[q])
    //   plane 9 + r  (r < 9)  the row weights of union row r, likewise
    //   plane 18              (r0 | c0 << 16, slot0 | slot1 << 16,
    //                          slot2 | slot3 << 16, 0): union origin in S and
    //                          the block-local node index of each slot
    // A node's weights are zero outside its own 8 x 8 window; slot 0xFFFF:
    // no node (zero weights).  Results are staged in the (now idle) warp
    // buffers, two blocks deep so that one barrier per block suffices.
    static_assert(W == 8 && FUS_UW == W + 1, "unit records hold 9 + 9 weights per node");
    const int nh = n_theta / 2;
    const int lbeg = (half == 0) ? 0 : nq0;
    const int nl = (half == 0) ? nq0 : nh - nq0;
    const int nblk = (half == 0) ? nblk0 : nblk1;
    const int gb0 = (half == 0) ? 0 : nblk0;
    float2 *Fout = Fpol + (size_t)img * n_xi * nh;
    float2 *stage0 = smz + SR * SLD;
    // t / nl as a multiply-high: exact for t < 2^32 / nl (nl >= 31 on this
    // path, so the multiplier does not overflow)
    const unsigned nl_magic = 0xFFFFFFFFu / (unsigned)nl + 1u;
    constexpr int GU = FUS_GU;   // the plan keeps a block's nodes within GN (one staging buffer)
    for (int b = 0; b < nblk; ++b) {
        const int2 tb = __ldg(&blocks[gb0 + b]);
        const int t0 = tb.x, cnt = tb.y;
        float2 *stage = stage0 + (b & 1) * GN;
        const float4 *rec = units + (size_t)(gb0 + b) * FUS_REC * GU;
        const int s = threadIdx.x;                 // one unit per thread
        const float4 meta = __ldg(&rec[18 * GU + s]);
        const unsigned s01 = __float_as_uint(meta.y), s23 = __float_as_uint(meta.z);
        const int sl[4] = {(int)(s01 & 0xFFFFu), (int)(s01 >> 16), (int)(s23 & 0xFFFFu), (int)(s23 >> 16)};
        if (sl[0] < cnt) {
            const int rc = __float_as_int(meta.x);
            const int r0 = rc & 0xFFFF, c0 = rc >> 16;
            float2 acc[FUS_NU];
#pragma unroll
            for (int n = 0; n < FUS_NU; ++n) acc[n] = make_float2(0.f, 0.f);
            if (r0 + FUS_UW > SR || c0 + FUS_UW > SLD) {
                ffb_flag(status, FFB_ERR_ARG);
            } else {
                float wx[FUS_UW][FUS_NU];
#pragma unroll
                for (int q = 0; q < FUS_UW; ++q) {
                    const float4 v = __ldg(&rec[q * GU + s]);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int n = 0; n < FUS_NU; ++n) wx[q][n] = vv[n];
                }
                // row by row: the 9 values of the union row, interpolated
                // along the row with each node's column weights, then
                // weighted by the node's row weight
                const float2 *base = S + r0 * SLD + c0;
#pragma unroll 1
                for (int r = 0; r < FUS_UW; ++r) {
                    const float4 wv = __ldg(&rec[(FUS_UW + r) * GU + s]);
                    const float wy[4] = {wv.x, wv.y, wv.z, wv.w};
                    const float2 *row = base + r * SLD;
                    float2 u[FUS_NU];
#pragma unroll
                    for (int n = 0; n < FUS_NU; ++n) u[n] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < FUS_UW; ++q) {
                        const float2 g = row[q];
#pragma unroll
                        for (int n = 0; n < FUS_NU; ++n) {
                            u[n].x = fmaf(wx[q][n], g.x, u[n].x);
                            u[n].y = fmaf(wx[q][n], g.y, u[n].y);
                        }
                    }
#pragma unroll
                    for (int n = 0; n < FUS_NU; ++n) {
                        acc[n].x = fmaf(wy[n], u[n].x, acc[n].x);
                        acc[n].y = fmaf(wy[n], u[n].y, acc[n].y);
                    }
                }
            }
#pragma unroll
            for (int n = 0; n < FUS_NU; ++n)
                if (sl[n] < cnt) stage[sl[n]] = acc[n];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += FUS_NT) {
            const int t = t0 + i;
            const int j = (int)__umulhi((unsigned)t, nl_magic);
            const int l = lbeg + (t - j * nl);
            if (planes) {
                // u and v as bf16 hi / lo planes [hi, lo][u, v][image][ring][l]
                // (the tensor-core ring DFT's operands)
                const float2 v = stage[i];
                const size_t o = ((size_t)img * n_xi + j) * nh + l;
                const __nv_bfloat16 uh = __float2bfloat16_rn(v.x), vh = __float2bfloat16_rn(v.y);
                planes[o] = uh;
                planes[(size_t)pstride + o] = vh;
                planes[2 * (size_t)pstride + o] = __float2bfloat16_rn(v.x - __bfloat162float(uh));
                planes[3 * (size_t)pstride + o] = __float2bfloat16_rn(v.y - __bfloat162float(vh));
            } else {
                Fout[(size_t)j * nh + l] = stage[i];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int N, int W>
static size_t fused_smem() {
    return sizeof(float2) * ((size_t)fus_rows(N, W) * fus_sld(N, W) + (size_t)FUS_WARPS * N);
}

// 1 when the cluster variant keeps every SM busy: clusters of two CTAs (one
// per SM) can occupy all SMs at once; FFB_FUSED_CLUSTER=0 in the environment
// at plan creation selects the plain variant
template <int N, int W>
static int fused_cluster_ok() {
    const char *ev = std::getenv("FFB_FUSED_CLUSTER");
    if (ev && ev[0] == '0') return 0;
    const size_t smem = fused_smem<N, W>();
    if (cudaFuncSetAttribute(k_grid_interp_half<N, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 0, ncl = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1024);
    cfg.blockDim = dim3(FUS_NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_grid_interp_half<N, W, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (2 * ncl >= sms) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Adjoint of phase 3 (step a10): spreading.  One CTA per (image, half): the
// half's polar values g (from the inverse ring DFT, layout of the polar
// buffer) are spread into the half grid held in shared memory with the
// forward's unit table, S[r0 + r][c0 + q] += sum_n wy_n[r] wx_n[q] g_n over
// the nodes of a unit (one shared-memory atomic per value of the 9 x 9 union
// and component; the unit order that keeps the forward's gathers on distinct
// banks does the same for these adds), and the half grid
// is then added into the extended grid Gext[m2 + h][m1 mod N] (global
// atomics: both halves overlap near m1 = 0 and m1 = +-N/2).  Gext is zeroed
// by the caller.  This is the transpose of phase 3 with the same weights, so
// the adjoint stays exact against the forward.
// ---------------------------------------------------------------------------
template <int N, int W>
__global__ void __launch_bounds__(FUS_NT, 1)
k_adj_spread_half(const float2 *__restrict__ Gpol, int n_xi, int n_theta, int nq0,
                  const float4 *__restrict__ units, const int2 *__restrict__ blocks, int nblk0, int nblk1,
                  float2 *__restrict__ Gext, int *status) {
    constexpr int H = (W + 1) / 2;
    constexpr int MH = fus_mh(N, W);
    constexpr int SLD = fus_sld(N, W);
    constexpr int SR = fus_rows(N, W);
    constexpr int GU = FUS_GU;
    static_assert(W == 8 && FUS_UW == W + 1, "unit records hold 9 + 9 weights per node");
    extern __shared__ float2 smz[];
    float *S = (float *)smz;                      // [SR][SLD] complex, as float pairs
    const int half = blockIdx.x;
    const int img = blockIdx.y;
    for (int i = threadIdx.x; i < SR * SLD; i += FUS_NT) smz[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int nh = n_theta / 2;
    const int lbeg = (half == 0) ? 0 : nq0;
    const int nl = (half == 0) ? nq0 : nh - nq0;
    const int nblk = (half == 0) ? nblk0 : nblk1;
    const int gb0 = (half == 0) ? 0 : nblk0;
    const float2 *Gp = Gpol + (size_t)img * n_xi * nh;
    const unsigned nl_magic = 0xFFFFFFFFu / (unsigned)nl + 1u;   // t / nl, as in phase 3
    // the polar value of the node in block slot sl (zero for an empty slot)
    auto value = [&](int t0, int cnt, int sl) {
        if (sl >= cnt) return make_float2(0.f, 0.f);
        const int t = t0 + sl;
        const int j = (int)__umulhi((unsigned)t, nl_magic);
        return __ldg(&Gp[(size_t)j * nh + lbeg + (t - j * nl)]);
    };
    for (int b = 0; b < nblk; ++b) {
        const int2 tb = __ldg(&blocks[gb0 + b]);
        const int t0 = tb.x, cnt = tb.y;
        const float4 *rec = units + (size_t)(gb0 + b) * FUS_REC * GU;
        const int s = threadIdx.x;                 // one unit per thread
        const float4 meta = __ldg(&rec[18 * GU + s]);
        const unsigned s01 = __float_as_uint(meta.y), s23 = __float_as_uint(meta.z);
        const int sl0 = (int)(s01 & 0xFFFFu);
        if (sl0 >= cnt) continue;
        const int rc = __float_as_int(meta.x);
        const int r0 = rc & 0xFFFF, c0 = rc >> 16;
        if (r0 + FUS_UW > SR || c0 + FUS_UW > SLD) {
            ffb_flag(status, FFB_ERR_ARG);
            continue;
        }
        const float2 v0 = value(t0, cnt, sl0), v1 = value(t0, cnt, (int)(s01 >> 16));
        const float2 v2 = value(t0, cnt, (int)(s23 & 0xFFFFu)), v3 = value(t0, cnt, (int)(s23 >> 16));
        float4 wx[FUS_UW];
#pragma unroll
        for (int q = 0; q < FUS_UW; ++q) wx[q] = __ldg(&rec[q * GU + s]);
        float *base = S + 2 * (r0 * SLD + c0);
        // S[r0 + r][c0 + q] += sum_n wy_n[r] wx_n[q] v_n: the transpose of the
        // forward's row-by-row interpolation, one shared atomic per grid
        // value and component
#pragma unroll 1
        for (int r = 0; r < FUS_UW; ++r) {
            const float4 wy = __ldg(&rec[(FUS_UW + r) * GU + s]);
            const float2 u0 = make_float2(wy.x * v0.x, wy.x * v0.y), u1 = make_float2(wy.y * v1.x, wy.y * v1.y);
            const float2 u2 = make_float2(wy.z * v2.x, wy.z * v2.y), u3 = make_float2(wy.w * v3.x, wy.w * v3.y);
            float *row = base + 2 * r * SLD;
#pragma unroll
            for (int q = 0; q < FUS_UW; ++q) {
                const float re = fmaf(wx[q].x, u0.x, fmaf(wx[q].y, u1.x, fmaf(wx[q].z, u2.x, wx[q].w * u3.x)));
                const float im = fmaf(wx[q].x, u0.y, fmaf(wx[q].y, u1.y, fmaf(wx[q].z, u2.y, wx[q].w * u3.y)));
                atomicAdd(&row[2 * q], re);
                atomicAdd(&row[2 * q + 1], im);
            }
        }
    }
    __syncthreads();
    // the half grid into Gext: row e is m2 = e - H (Gext's own offset), column
    // c is m1 = c + m1lo (the zero row and columns past MH are not copied)
    const int m1lo = (half == 0) ? -H : -(N / 2) - H;
    float2 *Gi = Gext + (size_t)img * MH * N;
    for (int i = threadIdx.x; i < MH * MH; i += FUS_NT) {
        const int e = i / MH, c = i - e * MH;
        const int col = (c + m1lo + N) & (N - 1);
        atomicAdd(&Gi[(size_t)e * N + col], smz[e * SLD + c]);
    }
}

int ffb_launch_fused_spread(ffb_plan_t p, const float2 *Gpol, int m, float2 *Gext, cudaStream_t s) {
    if (p->N != 256 && p->N != 128) return FFB_ERR_UNSUPPORTED;
    const int N = p->N;
    const size_t smem = sizeof(float2) * (size_t)fus_rows(N, 8) * fus_sld(N, 8);
    static int attr256 = 0, attr128 = 0;
    int &done = (N == 256) ? attr256 : attr128;
    const void *fn = (N == 256) ? (const void *)k_adj_spread_half<256, 8> : (const void *)k_adj_spread_half<128, 8>;
    if (done < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        done = (int)smem;
    }
    dim3 g(2, m);
    ProfScope ps(p, FFB_KC_ADJ_SPREAD, s);
    if (N == 256)
        k_adj_spread_half<256, 8><<<g, FUS_NT, smem, s>>>(Gpol, p->n_xi, p->n_theta, p->nq0, p->d_nodes,
                                                           p->d_node_blk, p->node_nblk[0], p->node_nblk[1], Gext,
                                                           p->d_status);
    else
        k_adj_spread_half<128, 8><<<g, FUS_NT, smem, s>>>(Gpol, p->n_xi, p->n_theta, p->nq0, p->d_nodes,
                                                           p->d_node_blk, p->node_nblk[0], p->node_nblk[1], Gext,
                                                           p->d_status);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// pdl: launched with programmatic serialization (the previous kernel in the
// stream is one of this library's and does not write the images)
template <int N, int W>
static int launch_fused(ffb_plan_t p, const float *d_images, int64_t i0, int m, float2 *Fpol, cudaStream_t s,
                        bool pdl, int64_t n_after, bool planes) {
    static int attr = 0, attr_cl = 0;
    const size_t smem = fused_smem<N, W>();
    const bool cl = p->fused == 2;
    int &done = cl ? attr_cl : attr;
    if (done < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(cl ? k_grid_interp_half<N, W, true> : k_grid_interp_half<N, W, false>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        done = (int)smem;
    }
    const float *img = d_images + (size_t)i0 * p->L * p->L;
    // images per wave at one CTA per SM and two per image (the N = 256
    // kernel; smaller grids run more CTAs per SM and the prefetch, a hint,
    // then lands on images already under way)
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int wave = sms / 2;
    ProfScope ps(p, FFB_KC_GRID_INTERP, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, m);
    cfg.blockDim = dim3(FUS_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (cl) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = 2;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    if (pdl) at[na++] = ffb_pdl_attr();
    cfg.attrs = at;
    cfg.numAttrs = na;
    int e = ffb_check_cuda(cudaLaunchKernelEx(&cfg, cl ? k_grid_interp_half<N, W, true> : k_grid_interp_half<N, W, false>,
                                              img, p->off, (const float *)p->d_corr, (const float2 *)p->d_twN,
                                              (const float2 *)p->d_twG, p->n_xi, p->n_theta, p->nq0, (const float4 *)p->d_nodes,
                                              (const int2 *)p->d_node_blk, p->node_nblk[0], p->node_nblk[1], Fpol,
                                              p->d_status, wave, (int)std::min<int64_t>(n_after, 1 << 20),
                                              planes ? (__nv_bfloat16 *)Fpol : (__nv_bfloat16 *)nullptr,
                                              (long long)p->chunk * p->n_xi * (p->n_theta / 2)));
    p->launches++;
    return e;
}

int ffb_fused_mode(ffb_plan_t p) {
    if (p->N == 256) return 1 + fused_cluster_ok<256, 8>();
    if (p->N == 128) return 1 + fused_cluster_ok<128, 8>();
    return 1;
}

bool ffb_fused_supported(ffb_plan_t p) {
    if (p->L * 2 != p->N || p->w != 8) return false;
    if (!(p->N == 128 || p->N == 256)) return false;
    if (!(p->n_theta == 128 || p->n_theta == 256 || p->n_theta == 512)) return false;
    if (p->k_max >= p->n_theta / 2) return false;
    if (p->L % 32) return false;
    const size_t smem = (p->N == 256) ? fused_smem<256, 8>() : fused_smem<128, 8>();
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return smem <= (size_t)optin;
}

// Units and blocks of phase 3 (see the file header).  For node t = j nl + l'
// of a half, p = N xi_j (cos theta_l, sin theta_l) in grid units, the window
// starts at m = ceil(p - W/2) and the weights are phi(f - b), f = p - m,
// b = 0..7, phi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) the ES kernel
// (Sec. III, type-2 NUFFT), in float64.  A block takes the longest run of
// consecutive nodes, at most GN, that groups into at most GU units.
// Grouping within a block: nodes sorted by (r0, c0); the first node not yet
// taken anchors a unit and takes up to three more untaken nodes whose window
// origins lie in the 2 x 2 box (r0 .. r0 + 1, c0 .. c0 + 1), in the order
// same origin, right, below, below right.  Units are ordered per half warp
// with distinct bank slots (union row * SLD + union column) mod 16: one unit
// from every nonempty slot, fullest slot first, then fill from the fullest.
static int build_units(int N, int W, double beta, int n_xi, int n_theta, const double *xi,
                       std::vector<float4> &rec, std::vector<int2> &blk, int nb[2]) {
    if (W != 8 || !(N == 128 || N == 256) || n_xi < 1 || n_theta < 4 || (n_theta & 1) || !xi)
        return FFB_ERR_UNSUPPORTED;
    const int H = (W + 1) / 2, SLD = fus_sld(N, W), MH = fus_mh(N, W), SR = fus_rows(N, W);
    const int GN = FUS_WARPS * N / 2, GU = FUS_GU;
    const int nh = n_theta / 2, nq0 = n_theta / 4 + 1;
    auto phi = [&](double x) {
        const double z = 2.0 * x / W, u = 1.0 - z * z;
        return (u > 0.0) ? std::exp(beta * (std::sqrt(u) - 1.0)) : 0.0;
    };
    auto bits = [](unsigned v) {
        float f;
        std::memcpy(&f, &v, sizeof f);
        return f;
    };
    struct Node {
        int r0, c0;
        double f1, f2;
    };
    struct Unit {
        int n;
        int idx[4];   // block-local node indices (FUS_NU used)
    };
    rec.clear();
    blk.clear();
    nb[0] = nb[1] = 0;
    for (int half = 0; half < 2; ++half) {
        const int lbeg = (half == 0) ? 0 : nq0;
        const int nl = (half == 0) ? nq0 : nh - nq0;
        const int npts = n_xi * nl;
        const int m1lo = (half == 0) ? -H : -(N / 2) - H;
        std::vector<Node> nd(npts);
        for (int t = 0; t < npts; ++t) {
            const int j = t / nl, l = lbeg + t % nl;
            const double th = 2.0 * M_PI * (double)l / (double)n_theta;
            const double p1 = N * xi[j] * std::cos(th), p2 = N * xi[j] * std::sin(th);
            const double m1 = std::ceil(p1 - 0.5 * W), m2 = std::ceil(p2 - 0.5 * W);
            const int c0 = (int)m1 - m1lo, r0 = (int)m2 + H;
            if (c0 < 0 || c0 + W > MH || r0 < 0 || r0 + W > MH) return FFB_ERR_UNSUPPORTED;
            nd[t] = {r0, c0, p1 - m1, p2 - m2};
        }
        // units of the nodes [t0, t1), node indices block-local
        auto group = [&](int t0, int t1) {
            const int n = t1 - t0;
            std::vector<int> ord(n);
            for (int i = 0; i < n; ++i) ord[i] = i;
            auto key = [&](int i) { return (int64_t)nd[t0 + i].r0 * 65536 + nd[t0 + i].c0; };
            std::sort(ord.begin(), ord.end(), [&](int x, int y) {
                const int64_t kx = key(x), ky = key(y);
                return (kx != ky) ? kx < ky : x < y;
            });
            std::vector<char> used(n, 0);
            std::vector<Unit> un;
            // position in ord of the first node at or after origin (r, c)
            auto first_at = [&](int r, int c) {
                const int64_t k = (int64_t)r * 65536 + c;
                return (int)(std::lower_bound(ord.begin(), ord.end(), k,
                                              [&](int i, int64_t kk) { return key(i) < kk; }) -
                             ord.begin());
            };
            for (int a = 0; a < n; ++a) {
                const int ia = ord[a];
                if (used[ia]) continue;
                Unit u{1, {ia, -1, -1, -1}};
                used[ia] = 1;
                const int r = nd[t0 + ia].r0, c = nd[t0 + ia].c0;
                const int cells[4][2] = {{r, c}, {r, c + 1}, {r + 1, c}, {r + 1, c + 1}};
                for (int cc = 0; cc < 4 && u.n < FUS_NU; ++cc) {
                    const int64_t k = (int64_t)cells[cc][0] * 65536 + cells[cc][1];
                    for (int p = first_at(cells[cc][0], cells[cc][1]); p < n && key(ord[p]) == k && u.n < FUS_NU; ++p)
                        if (!used[ord[p]]) {
                            used[ord[p]] = 1;
                            u.idx[u.n++] = ord[p];
                        }
                }
                un.push_back(u);
            }
            return un;
        };
        for (int t0 = 0; t0 < npts;) {
            // a long node range whose units fit: full blocks of GU units (the
            // search keeps only ranges that were checked to fit)
            int lo = t0 + 1, hi = std::min(npts, t0 + GN);
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if ((int)group(t0, mid).size() <= GU) lo = mid;
                else hi = mid - 1;
            }
            const int t1 = lo;
            std::vector<Unit> un = group(t0, t1);
            const int cnt = t1 - t0;
            if ((int)un.size() > GU) return FFB_ERR_UNSUPPORTED;
            blk.push_back(make_int2(t0, cnt));
            const size_t base = rec.size();
            rec.resize(base + (size_t)FUS_REC * GU, make_float4(0.f, 0.f, 0.f, 0.f));
            float4 *R = rec.data() + base;
            for (int sl = 0; sl < GU; ++sl) R[18 * GU + sl] = make_float4(0.f, bits(0xFFFFFFFFu), bits(0xFFFFFFFFu), 0.f);
            // union origin of each unit: the box origin (minimum row and column
            // of its nodes), or one row / column earlier where every node sits
            // in the box's first row / column and the union still fits,
            // chosen to even out the bank slots: fixed units first, then each
            // movable one into its emptiest candidate slot
            const int nu = (int)un.size();
            std::vector<int> urow(nu), ucol(nu);
            int cnt16[16] = {};
            std::vector<std::vector<std::pair<int, int>>> cand(nu);
            for (int u = 0; u < nu; ++u) {
                int rmin = 1 << 30, cmin = 1 << 30, rmax = -1, cmax = -1;
                for (int i = 0; i < un[u].n; ++i) {
                    const Node &v = nd[t0 + un[u].idx[i]];
                    rmin = std::min(rmin, v.r0);
                    rmax = std::max(rmax, v.r0);
                    cmin = std::min(cmin, v.c0);
                    cmax = std::max(cmax, v.c0);
                }
                const bool mr = (rmax == rmin) && rmin >= 1, mc = (cmax == cmin) && cmin >= 1;
                cand[u].push_back({rmin, cmin});
                if (mc) cand[u].push_back({rmin, cmin - 1});
                if (mr) cand[u].push_back({rmin - 1, cmin});
                if (mr && mc) cand[u].push_back({rmin - 1, cmin - 1});
                urow[u] = rmin;
                ucol[u] = cmin;
                if (cand[u].size() == 1) cnt16[(rmin * SLD + cmin) & 15]++;
            }
            for (int u = 0; u < nu; ++u) {
                if (cand[u].size() == 1) continue;
                int best = 0;
                for (int k = 1; k < (int)cand[u].size(); ++k)
                    if (cnt16[(cand[u][k].first * SLD + cand[u][k].second) & 15] <
                        cnt16[(cand[u][best].first * SLD + cand[u][best].second) & 15])
                        best = k;
                urow[u] = cand[u][best].first;
                ucol[u] = cand[u][best].second;
                cnt16[(urow[u] * SLD + ucol[u]) & 15]++;
            }
            std::vector<int> bucket[16];
            for (int u = nu - 1; u >= 0; --u) bucket[(urow[u] * SLD + ucol[u]) & 15].push_back(u);
            int pos = 0;
            auto put = [&](int u) {
                const int ru = urow[u], cu = ucol[u];
                if (ru < 0 || cu < 0 || ru + FUS_UW > SR || cu + FUS_UW > SLD) return false;
                float wx[FUS_UW][4] = {}, wy[FUS_UW][4] = {};
                unsigned slot[4] = {0xFFFFu, 0xFFFFu, 0xFFFFu, 0xFFFFu};
                for (int i = 0; i < un[u].n; ++i) {
                    const Node &v = nd[t0 + un[u].idx[i]];
                    const int dr = v.r0 - ru, dc = v.c0 - cu;   // 0 or 1
                    for (int q = 0; q < W; ++q) {
                        wx[dc + q][i] = (float)phi(v.f1 - q);
                        wy[dr + q][i] = (float)phi(v.f2 - q);
                    }
                    slot[i] = (unsigned)un[u].idx[i];
                }
                for (int q = 0; q < FUS_UW; ++q) {
                    R[q * GU + pos] = make_float4(wx[q][0], wx[q][1], wx[q][2], wx[q][3]);
                    R[(FUS_UW + q) * GU + pos] = make_float4(wy[q][0], wy[q][1], wy[q][2], wy[q][3]);
                }
                // slots as unsigned halves (0xFFFF: none); the kernels decode
                // them with logical shifts
                R[18 * GU + pos] = make_float4(bits((unsigned)ru | ((unsigned)cu << 16)),
                                               bits(slot[0] | (slot[1] << 16)), bits(slot[2] | (slot[3] << 16)), 0.f);
                ++pos;
                return true;
            };
            while (pos < nu) {
                int order[16];
                for (int r = 0; r < 16; ++r) order[r] = r;
                std::stable_sort(order, order + 16, [&](int x, int y) { return bucket[x].size() > bucket[y].size(); });
                int taken = 0;
                for (int r : order) {
                    if (bucket[r].empty()) continue;
                    if (!put(bucket[r].back())) return FFB_ERR_UNSUPPORTED;
                    bucket[r].pop_back();
                    ++taken;
                }
                while (taken < 16 && pos < nu) {
                    int rb = 0;
                    for (int r = 1; r < 16; ++r)
                        if (bucket[r].size() > bucket[rb].size()) rb = r;
                    if (!put(bucket[rb].back())) return FFB_ERR_UNSUPPORTED;
                    bucket[rb].pop_back();
                    ++taken;
                }
            }
            ++nb[half];
            t0 = t1;
        }
    }
    return FFB_OK;
}

int ffb_fused_prepare(ffb_plan_t p, cudaStream_t s) {
    const int N = p->N;
    std::vector<double> xi(p->n_xi);
    int e = ffb_check_cuda(cudaMemcpyAsync(xi.data(), p->d_xi, sizeof(double) * p->n_xi, cudaMemcpyDeviceToHost, s));
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (e) return e;
    std::vector<float4> rec;
    std::vector<int2> blk;
    int nb[2] = {0, 0};
    if ((e = build_units(N, p->w, p->beta, p->n_xi, p->n_theta, xi.data(), rec, blk, nb))) return e;
    // FFT twiddles W_N^{j k1} as [k1][j] (k1 < N / 32, j < 32: the whole-warp
    // FFT), then at N = 256 as [k1][j] (k1, j < 16: the half-warp FFT), from
    // float64
    {
        const int MG = N / 32;
        std::vector<float2> twg((size_t)MG * 32 + (N == 256 ? 256 : 0));
        for (int k1 = 0; k1 < MG; ++k1)
            for (int j = 0; j < 32; ++j) {
                const double a = -2.0 * M_PI * (double)((j * k1) % N) / (double)N;
                twg[(size_t)k1 * 32 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        if (N == 256)
            for (int k1 = 0; k1 < 16; ++k1)
                for (int j = 0; j < 16; ++j) {
                    const double a = -2.0 * M_PI * (double)((j * k1) % N) / (double)N;
                    twg[(size_t)N + k1 * 16 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        if (p->d_twG) cudaFree(p->d_twG);
        p->d_twG = nullptr;
        e = ffb_check_cuda(cudaMalloc((void **)&p->d_twG, sizeof(float2) * twg.size()));
        if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_twG, twg.data(), sizeof(float2) * twg.size(),
                                                   cudaMemcpyHostToDevice, s));
        if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
        if (e) return e;
    }
    if (p->d_nodes) cudaFree(p->d_nodes);
    if (p->d_node_blk) cudaFree(p->d_node_blk);
    p->d_nodes = nullptr;
    p->d_node_blk = nullptr;
    e = ffb_check_cuda(cudaMalloc((void **)&p->d_nodes, sizeof(float4) * rec.size()));
    if (!e) e = ffb_check_cuda(cudaMalloc((void **)&p->d_node_blk, sizeof(int2) * blk.size()));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_nodes, rec.data(), sizeof(float4) * rec.size(),
                                               cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_node_blk, blk.data(), sizeof(int2) * blk.size(),
                                               cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    p->node_nblk[0] = nb[0];
    p->node_nblk[1] = nb[1];
    return e;
}

extern "C" int ffb_interp_units(int N, int w, double beta, int n_xi, int n_theta, const double *h_xi,
                                int64_t *h_counts, float *h_rec, int *h_blk) {
    if (!h_counts || !h_xi || n_xi < 1 || n_theta < 4 || !(beta > 0.0)) return FFB_ERR_ARG;
    std::vector<float4> rec;
    std::vector<int2> blk;
    int nb[2] = {0, 0};
    const int e = build_units(N, w, beta, n_xi, n_theta, h_xi, rec, blk, nb);
    if (e) return e;
    h_counts[0] = (int64_t)rec.size();
    h_counts[1] = (int64_t)blk.size();
    h_counts[2] = nb[0];
    h_counts[3] = nb[1];
    h_counts[4] = FUS_GU;
    h_counts[5] = fus_mh(N, w);
    h_counts[6] = fus_sld(N, w);
    h_counts[7] = FUS_REC;
    h_counts[8] = FUS_NU;
    if (h_rec) std::memcpy(h_rec, rec.data(), sizeof(float4) * rec.size());
    if (h_blk) std::memcpy(h_blk, blk.data(), sizeof(int2) * blk.size());
    return FFB_OK;
}

int ffb_launch_fused_polar(ffb_plan_t p, const float *d_images, int64_t i0, int m, float2 *Fpol, cudaStream_t s,
                           bool pdl, int64_t n_after, bool planes) {
    if (planes && Fpol != p->d_Fpol) return FFB_ERR_ARG;   // the plane stride is the plan's chunk
    if (p->N == 256) return launch_fused<256, 8>(p, d_images, i0, m, Fpol, s, pdl, n_after, planes);
    if (p->N == 128) return launch_fused<128, 8>(p, d_images, i0, m, Fpol, s, pdl, n_after, planes);
    return FFB_ERR_UNSUPPORTED;
}
