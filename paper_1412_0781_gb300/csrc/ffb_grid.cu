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
// Phase 1  rows: for pixel rows a1 (two per complex FFT), the length-N DFT
//          over i2 of I(i) corr(i1) corr(i2) placed at i2 mod N; the outputs
//          m2 in [-h, N/2 + h] are stored in column a1 of S[m2 + h][.].
// Phase 2  columns: for each m2 row of S, the length-N DFT over i1 (entries
//          placed at i1 mod N); the half's m1 range overwrites the row in
//          place (the row is read completely before it is written).
// Phase 3  interpolation of the half's nodes from S (w x w taps of the ES
//          kernel with weights from the plan), the result written to the
//          polar buffer F[img][j][l], l < n_theta/2.
// The ring FFT (ffb_ring.cu) then completes every half ring with
// F(theta + pi) = conj F(theta) and takes the length-n_theta FFT of Eq. 1DFFT.
//
// Phases 1 and 2 are the same for both halves.  Where clusters of two CTAs
// fill the GPU, the two CTAs of an image form one and split them: each
// transforms half of the pixel-row pairs and half of the S rows, and sends
// the peer what it needs through distributed shared memory (contiguous row
// segments after phase 1, the peer's column range of every row it
// transformed in phase 2).
//
// Node order in phase 3.  A node gathers the W x W window of S at
// S[r0][c0] (W = 8).  Two nodes with the same r0 and window origins c0, c0 + d
// (d in {0, 1}) form a unit: one thread reads the 8 x 9 union of their
// windows once and forms both results, 36 gathers per node instead of 64
// (phase 3 is bound by the shared-memory pipe).  One 8-byte load of a half
// warp takes a single wavefront when the 16 unit origins r0 * SLD + c0 fall in
// distinct 8-byte bank slots (the origin mod 16) or coincide, so the units are
// ordered into half warps with distinct slots; a unit whose nodes share their
// column origin (or a single node) may start its union one column to the
// left, which the plan uses to even out the slots' unit counts.  Everything here depends on
// the geometry alone and is built by the plan in float64
// (ffb_fused_prepare): blocks of consecutive nodes t = j nl + l, at most
// FUS_GU units each, and per unit the origin, both
// nodes' 8 row weights and 9 column weights over the union (144 bytes, about
// 2.6 MB at N = 256, read from L2 by every CTA).  The kernel stages a block's
// results in shared memory and stores them in natural order.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ffb_fft.cuh"

#define FUS_WARPS 32                 // warps per CTA, each with an N-entry FFT buffer
#define FUS_NT (32 * FUS_WARPS)      // threads per CTA
#define FUS_GU 2048   // units per phase-3 block (at most; two per thread)
#define FUS_REC 9     // float4 fields of a unit record

// rows of the shared-memory grid block and its row pitch (complex entries):
// MH (odd) columns hold the half plane, two more zero columns let a unit's
// 9-column union start at the last window origin; the pitch stays odd
__host__ __device__ constexpr int fus_mh(int N, int W) { return N / 2 + 1 + 2 * ((W + 1) / 2); }
__host__ __device__ constexpr int fus_sld(int N, int W) { return fus_mh(N, W) + 2; }

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
                   float2 *__restrict__ Fpol, int *status) {
    constexpr int L = N / 2;
    constexpr int H = (W + 1) / 2;
    constexpr int MH = fus_mh(N, W);              // rows of S (m2 + h)
    constexpr int SLD = fus_sld(N, W);            // row length of S
    constexpr int GN = FUS_WARPS * N / 2;         // nodes per block at most (two staged blocks)
    extern __shared__ float2 smz[];
    float2 *S = smz;                               // [MH][SLD]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *buf = smz + MH * SLD + warp * N;   // this warp's FFT buffer
    const int half = blockIdx.x;
    const int img = blockIdx.y;
    const float *im = images + (size_t)img * L * L;
    pdl_trigger();
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

    // the polar buffer may still be read by the previous kernel (the ring FFT
    // of the previous chunk) when this launch started early
    pdl_wait();

    // ---- phase 3: interpolation of this half's nodes -----------------------
    // block b of the half covers the nodes t in [t0, t0 + cnt);
    // unit record s holds, as FUS_REC planes of FUS_GU float4,
    //   0, 1  row weights of node A    2, 3  row weights of node B
    //   4, 5  column weights of A, columns 0..7 of the union; 8.w: column 8
    //   6, 7  column weights of B, columns 0..7; 8.x: column 8
    //   8.y   r0 | c0 << 16 (union origin in S)   8.z  slotA | slotB << 16
    // slots index the block's nodes (0xFFFF: none; node B of a single unit
    // carries zero weights).  Results are staged in the (now idle) warp
    // buffers, two blocks deep so that one barrier per block suffices.
    static_assert(W == 8, "unit records hold 8 + 8 row and 9 + 9 column weights");
    const int nh = n_theta / 2;
    const int lbeg = (half == 0) ? 0 : nq0;
    const int nl = (half == 0) ? nq0 : nh - nq0;
    const int nblk = (half == 0) ? nblk0 : nblk1;
    const int gb0 = (half == 0) ? 0 : nblk0;
    float2 *Fout = Fpol + (size_t)img * n_xi * nh;
    float2 *stage0 = smz + MH * SLD;
    // t / nl as a multiply-high: exact for t < 2^32 / nl (nl >= 31 on this
    // path, so the multiplier does not overflow)
    const unsigned nl_magic = 0xFFFFFFFFu / (unsigned)nl + 1u;
    constexpr int GU = (FUS_GU < GN / 2) ? FUS_GU : GN / 2;   // units per block
    for (int b = 0; b < nblk; ++b) {
        const int2 tb = __ldg(&blocks[gb0 + b]);
        const int t0 = tb.x, cnt = tb.y;
        float2 *stage = stage0 + (b & 1) * GN;
        const float4 *rec = units + (size_t)(gb0 + b) * FUS_REC * GU;
#pragma unroll 1
        for (int s = threadIdx.x; s < GU; s += FUS_NT) {
            const float4 meta = __ldg(&rec[8 * GU + s]);
            const int locs = __float_as_int(meta.z);
            const int la = locs & 0xFFFF, lb = (int)((unsigned)locs >> 16);   // 0xFFFF: no node B
            if (la >= cnt) continue;
            const int rc = __float_as_int(meta.y);
            const int r0 = rc & 0xFFFF, c0 = rc >> 16;
            const float4 xa0 = __ldg(&rec[4 * GU + s]), xa1 = __ldg(&rec[5 * GU + s]);
            const float4 xb0 = __ldg(&rec[6 * GU + s]), xb1 = __ldg(&rec[7 * GU + s]);
            if (r0 + W > MH || c0 + W + 1 > SLD) {
                ffb_flag(status, FFB_ERR_ARG);
                stage[la] = make_float2(0.f, 0.f);
                if (lb < cnt) stage[lb] = make_float2(0.f, 0.f);
                continue;
            }
            const float wxa[9] = {xa0.x, xa0.y, xa0.z, xa0.w, xa1.x, xa1.y, xa1.z, xa1.w, meta.w};
            const float wxb[9] = {xb0.x, xb0.y, xb0.z, xb0.w, xb1.x, xb1.y, xb1.z, xb1.w, meta.x};
            // row by row: the 9 values of the union row, interpolated along
            // the row with each node's column weights, then weighted by the
            // node's row weight (rows 0..3, then 4..7, four row weights of
            // each node at a time)
            const float2 *base = S + r0 * SLD + c0;
            float2 aa = make_float2(0.f, 0.f), ab = make_float2(0.f, 0.f);
#pragma unroll
            for (int h4 = 0; h4 < 2; ++h4) {
                const float4 ya = __ldg(&rec[h4 * GU + s]), yb = __ldg(&rec[(2 + h4) * GU + s]);
                const float wya[4] = {ya.x, ya.y, ya.z, ya.w};
                const float wyb[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
                for (int b4 = 0; b4 < 4; ++b4) {
                    const float2 *row = base + (4 * h4 + b4) * SLD;
                    float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q <= W; ++q) {
                        const float2 g = row[q];
                        ra.x = fmaf(wxa[q], g.x, ra.x);
                        ra.y = fmaf(wxa[q], g.y, ra.y);
                        rb.x = fmaf(wxb[q], g.x, rb.x);
                        rb.y = fmaf(wxb[q], g.y, rb.y);
                    }
                    aa.x = fmaf(wya[b4], ra.x, aa.x);
                    aa.y = fmaf(wya[b4], ra.y, aa.y);
                    ab.x = fmaf(wyb[b4], rb.x, ab.x);
                    ab.y = fmaf(wyb[b4], rb.y, ab.y);
                }
            }
            stage[la] = aa;
            if (lb < cnt) stage[lb] = ab;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += FUS_NT) {
            const int t = t0 + i;
            const int j = (int)__umulhi((unsigned)t, nl_magic);
            const int l = lbeg + (t - j * nl);
            Fout[(size_t)j * nh + l] = stage[i];
        }
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int N, int W>
static size_t fused_smem() {
    return sizeof(float2) * ((size_t)fus_mh(N, W) * fus_sld(N, W) + (size_t)FUS_WARPS * N);
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
// forward's unit table, S[r0 + b][c0 + q] += wy_b wx_q g for both nodes of a
// unit (shared-memory atomics; the unit order that keeps the forward's
// gathers on distinct banks does the same for these adds), and the half grid
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
    constexpr int GN = FUS_WARPS * N / 2;
    constexpr int GU = (FUS_GU < GN / 2) ? FUS_GU : GN / 2;
    static_assert(W == 8, "unit records hold 8 + 8 row and 9 + 9 column weights");
    extern __shared__ float2 smz[];
    float *S = (float *)smz;                      // [MH][SLD] complex, as float pairs
    const int half = blockIdx.x;
    const int img = blockIdx.y;
    for (int i = threadIdx.x; i < MH * SLD; i += FUS_NT) smz[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int nh = n_theta / 2;
    const int lbeg = (half == 0) ? 0 : nq0;
    const int nl = (half == 0) ? nq0 : nh - nq0;
    const int nblk = (half == 0) ? nblk0 : nblk1;
    const int gb0 = (half == 0) ? 0 : nblk0;
    const float2 *Gp = Gpol + (size_t)img * n_xi * nh;
    const unsigned nl_magic = 0xFFFFFFFFu / (unsigned)nl + 1u;   // t / nl, as in phase 3
    for (int b = 0; b < nblk; ++b) {
        const int2 tb = __ldg(&blocks[gb0 + b]);
        const int t0 = tb.x, cnt = tb.y;
        const float4 *rec = units + (size_t)(gb0 + b) * FUS_REC * GU;
        for (int s = threadIdx.x; s < GU; s += FUS_NT) {
            const float4 meta = __ldg(&rec[8 * GU + s]);
            const int locs = __float_as_int(meta.z);
            const int la = locs & 0xFFFF, lb = (int)((unsigned)locs >> 16);   // 0xFFFF: no node B
            if (la >= cnt) continue;
            const int rc = __float_as_int(meta.y);
            const int r0 = rc & 0xFFFF, c0 = rc >> 16;
            if (r0 + W > MH || c0 + W + 1 > SLD) {
                ffb_flag(status, FFB_ERR_ARG);
                continue;
            }
            const int ta = t0 + la;
            const int ja = (int)__umulhi((unsigned)ta, nl_magic);
            const float2 va = __ldg(&Gp[(size_t)ja * nh + lbeg + (ta - ja * nl)]);
            float2 vb = make_float2(0.f, 0.f);
            if (lb < cnt) {
                const int tbn = t0 + lb;
                const int jb = (int)__umulhi((unsigned)tbn, nl_magic);
                vb = __ldg(&Gp[(size_t)jb * nh + lbeg + (tbn - jb * nl)]);
            }
            const float4 xa0 = __ldg(&rec[4 * GU + s]), xa1 = __ldg(&rec[5 * GU + s]);
            const float4 xb0 = __ldg(&rec[6 * GU + s]), xb1 = __ldg(&rec[7 * GU + s]);
            const float wxa[9] = {xa0.x, xa0.y, xa0.z, xa0.w, xa1.x, xa1.y, xa1.z, xa1.w, meta.w};
            const float wxb[9] = {xb0.x, xb0.y, xb0.z, xb0.w, xb1.x, xb1.y, xb1.z, xb1.w, meta.x};
            float *base = S + 2 * (r0 * SLD + c0);
#pragma unroll
            for (int h4 = 0; h4 < 2; ++h4) {
                const float4 ya = __ldg(&rec[h4 * GU + s]), yb = __ldg(&rec[(2 + h4) * GU + s]);
                const float wya[4] = {ya.x, ya.y, ya.z, ya.w};
                const float wyb[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
                for (int b4 = 0; b4 < 4; ++b4) {
                    const float2 ua = make_float2(wya[b4] * va.x, wya[b4] * va.y);
                    const float2 ub = make_float2(wyb[b4] * vb.x, wyb[b4] * vb.y);
                    float *row = base + 2 * (4 * h4 + b4) * SLD;
#pragma unroll
                    for (int q = 0; q <= W; ++q) {
                        atomicAdd(&row[2 * q], fmaf(wxa[q], ua.x, wxb[q] * ub.x));
                        atomicAdd(&row[2 * q + 1], fmaf(wxa[q], ua.y, wxb[q] * ub.y));
                    }
                }
            }
        }
    }
    __syncthreads();
    // the half grid into Gext: row e is m2 = e - H (Gext's own offset), column
    // c is m1 = c + m1lo
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
    const size_t smem = sizeof(float2) * (size_t)fus_mh(N, 8) * fus_sld(N, 8);
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
                        bool pdl) {
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
                                              p->d_status));
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
// consecutive nodes, at most GN, that pairs into at most GU units.  Pairing within a
// block: nodes sorted by (r0, c0), each joined with the next when that has the
// same r0 and c0 at most one larger (left to right, a maximum matching of
// this interval structure); the rest are single units.  Units are ordered per
// half warp with distinct bank slots (r0 SLD + c0) mod 16: one unit from every
// nonempty slot, fullest slot first, then fill from the fullest.
static int build_units(int N, int W, double beta, int n_xi, int n_theta, const double *xi,
                       std::vector<float4> &rec, std::vector<int2> &blk, int nb[2]) {
    if (W != 8 || !(N == 128 || N == 256) || n_xi < 1 || n_theta < 4 || (n_theta & 1) || !xi)
        return FFB_ERR_UNSUPPORTED;
    const int H = (W + 1) / 2, SLD = fus_sld(N, W), MH = fus_mh(N, W);
    const int GN = FUS_WARPS * N / 2, GU = std::min(FUS_GU, GN / 2);
    const int nh = n_theta / 2, nq0 = n_theta / 4 + 1;
    auto phi = [&](double x) {
        const double z = 2.0 * x / W, u = 1.0 - z * z;
        return (u > 0.0) ? std::exp(beta * (std::sqrt(u) - 1.0)) : 0.0;
    };
    auto bits = [](int v) {
        float f;
        std::memcpy(&f, &v, sizeof f);
        return f;
    };
    struct Node {
        int r0, c0;
        double f1, f2;
    };
    rec.clear();
    blk.clear();
    nb[0] = nb[1] = 0;
    for (int half = 0; half < 2; ++half) {
        const int lbeg = (half == 0) ? 0 : nq0;
        const int nl = (half == 0) ? nq0 : nh - nq0;
        const int npts = n_xi * nl;
        const int m1lo = (half == 0) ? -H : -(N / 2) - H;
        if (nl > GN) return FFB_ERR_UNSUPPORTED;
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
        // units of the nodes [t0, t1): (A, B) block-local, B = -1 for a single
        auto pair_up = [&](int t0, int t1) {
            std::vector<int> ord(t1 - t0);
            for (int i = 0; i < t1 - t0; ++i) ord[i] = i;
            std::sort(ord.begin(), ord.end(), [&](int x, int y) {
                const Node &u = nd[t0 + x], &v = nd[t0 + y];
                return (u.r0 != v.r0) ? u.r0 < v.r0 : (u.c0 != v.c0) ? u.c0 < v.c0 : x < y;
            });
            std::vector<std::pair<int, int>> un;
            for (size_t i = 0; i < ord.size();) {
                if (i + 1 < ord.size()) {
                    const Node &u = nd[t0 + ord[i]], &v = nd[t0 + ord[i + 1]];
                    if (u.r0 == v.r0 && v.c0 - u.c0 <= 1) {
                        un.push_back({ord[i], ord[i + 1]});
                        i += 2;
                        continue;
                    }
                }
                un.push_back({ord[i], -1});
                ++i;
            }
            return un;
        };
        for (int t0 = 0; t0 < npts;) {
            // the longest node range whose units fit (the unit count of a
            // range never decreases as it grows): full blocks of GU units
            int lo = t0 + 1, hi = std::min(npts, t0 + GN);
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if ((int)pair_up(t0, mid).size() <= GU) lo = mid;
                else hi = mid - 1;
            }
            const int t1 = lo;
            std::vector<std::pair<int, int>> un = pair_up(t0, t1);
            const int cnt = t1 - t0;
            blk.push_back(make_int2(t0, cnt));
            const size_t base = rec.size();
            rec.resize(base + (size_t)FUS_REC * GU, make_float4(0.f, 0.f, 0.f, 0.f));
            float4 *R = rec.data() + base;
            for (int sl = 0; sl < GU; ++sl) R[8 * GU + sl] = make_float4(0.f, 0.f, bits((int)0xFFFFFFFFu), 0.f);
            // union origin of each unit: A's window origin, or one column to
            // its left where both nodes' windows still fit (the same column
            // origin, or a single node), chosen to even out the bank slots:
            // the fixed units first, then each movable one into the emptier
            // of its two slots
            const int nu0 = (int)un.size();
            std::vector<int> ucol(nu0);
            int cnt16[16] = {};
            std::vector<char> movable(nu0);
            for (int u = 0; u < nu0; ++u) {
                const Node &a = nd[t0 + un[u].first];
                movable[u] = (un[u].second < 0 || nd[t0 + un[u].second].c0 == a.c0) && a.c0 >= 1;
                ucol[u] = a.c0;
                if (!movable[u]) cnt16[(a.r0 * SLD + a.c0) & 15]++;
            }
            for (int u = 0; u < nu0; ++u) {
                if (!movable[u]) continue;
                const Node &a = nd[t0 + un[u].first];
                const int s0 = (a.r0 * SLD + a.c0) & 15, s1 = (s0 + 15) & 15;
                if (cnt16[s1] < cnt16[s0]) ucol[u] = a.c0 - 1;
                cnt16[(a.r0 * SLD + ucol[u]) & 15]++;
            }
            std::vector<int> bucket[16];
            for (int u = nu0 - 1; u >= 0; --u) {
                const Node &a = nd[t0 + un[u].first];
                bucket[(a.r0 * SLD + ucol[u]) & 15].push_back(u);
            }
            int pos = 0;
            auto put = [&](int u) {
                const int ia = un[u].first, ib = un[u].second;
                const Node &a = nd[t0 + ia];
                const int cu = ucol[u];
                float w[36] = {};   // row A (8), row B (8), column A (9), column B (9)
                for (int q = 0; q < W; ++q) {
                    w[q] = (float)phi(a.f2 - q);
                    w[16 + (a.c0 - cu) + q] = (float)phi(a.f1 - q);
                }
                if (ib >= 0) {
                    const Node &bn = nd[t0 + ib];
                    const int d = bn.c0 - cu;   // 0, 1
                    for (int q = 0; q < W; ++q) {
                        w[8 + q] = (float)phi(bn.f2 - q);
                        w[25 + d + q] = (float)phi(bn.f1 - q);
                    }
                }
                // fields: rows A, rows B, columns A 0..7, columns B 0..7,
                // (column B 8, origin, slots, column A 8)
                const float4 f0 = make_float4(w[0], w[1], w[2], w[3]), f1 = make_float4(w[4], w[5], w[6], w[7]);
                const float4 f2 = make_float4(w[8], w[9], w[10], w[11]), f3 = make_float4(w[12], w[13], w[14], w[15]);
                const float4 f4 = make_float4(w[16], w[17], w[18], w[19]), f5 = make_float4(w[20], w[21], w[22], w[23]);
                const float4 f6 = make_float4(w[25], w[26], w[27], w[28]), f7 = make_float4(w[29], w[30], w[31], w[32]);
                R[0 * GU + pos] = f0;
                R[1 * GU + pos] = f1;
                R[2 * GU + pos] = f2;
                R[3 * GU + pos] = f3;
                R[4 * GU + pos] = f4;
                R[5 * GU + pos] = f5;
                R[6 * GU + pos] = f6;
                R[7 * GU + pos] = f7;
                // slots as unsigned halves (0xFFFF: no node B); the kernels
                // decode them with logical shifts
                const unsigned locs = (unsigned)ia | ((unsigned)(ib >= 0 ? ib : 0xFFFF) << 16);
                R[8 * GU + pos] = make_float4(w[33], bits(a.r0 | (cu << 16)), bits((int)locs), w[24]);
                ++pos;
            };
            const int nu = (int)un.size();
            while (pos < nu) {
                int order[16];
                for (int r = 0; r < 16; ++r) order[r] = r;
                std::stable_sort(order, order + 16, [&](int x, int y) { return bucket[x].size() > bucket[y].size(); });
                int taken = 0;
                for (int r : order) {
                    if (bucket[r].empty()) continue;
                    put(bucket[r].back());
                    bucket[r].pop_back();
                    ++taken;
                }
                while (taken < 16 && pos < nu) {
                    int rb = 0;
                    for (int r = 1; r < 16; ++r)
                        if (bucket[r].size() > bucket[rb].size()) rb = r;
                    put(bucket[rb].back());
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
    // FFT twiddles W_N^{j k1} as [k1][j] (k1 < N / 32, j < 32), from float64
    {
        const int MG = N / 32;
        std::vector<float2> twg((size_t)MG * 32);
        for (int k1 = 0; k1 < MG; ++k1)
            for (int j = 0; j < 32; ++j) {
                const double a = -2.0 * M_PI * (double)((j * k1) % N) / (double)N;
                twg[(size_t)k1 * 32 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
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
    h_counts[4] = std::min(FUS_GU, FUS_WARPS * N / 4);
    h_counts[5] = fus_mh(N, w);
    h_counts[6] = fus_sld(N, w);
    if (h_rec) std::memcpy(h_rec, rec.data(), sizeof(float4) * rec.size());
    if (h_blk) std::memcpy(h_blk, blk.data(), sizeof(int2) * blk.size());
    return FFB_OK;
}

int ffb_launch_fused_polar(ffb_plan_t p, const float *d_images, int64_t i0, int m, float2 *Fpol, cudaStream_t s,
                           bool pdl) {
    if (p->N == 256) return launch_fused<256, 8>(p, d_images, i0, m, Fpol, s, pdl);
    if (p->N == 128) return launch_fused<128, 8>(p, d_images, i0, m, Fpol, s, pdl);
    return FFB_ERR_UNSUPPORTED;
}
