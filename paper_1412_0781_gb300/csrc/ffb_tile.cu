// ffb_tile.cu -- step a3 (the interpolation of the type-2 NUFFT of Eq.
// nufft onto the polar nodes) for the plans whose oversampled half grid does
// not fit in one SM's shared memory: the separate-kernel path (k_rows and
// k_cols write the half grid G[Mh][N] of each image to global memory).
//
// The half grid is cut into tiles of TIL_TR x TIL_TC window origins.  A node
// belongs to the tile that holds its window origin (r0, u) = (m2 + h,
// m1 + N/2 + h) (row of G, unwrapped column); the nodes of a tile are grouped
// into units of up to four nodes whose origins lie in one 2 x 2 box, read
// from the 9 x 9 union of their windows, exactly as in the shared-memory grid
// kernel (ffb_grid.cu), and a tile's units are split into blocks of at most
// one unit per thread.  One CTA per (block, image) copies its tile plus the
// 8-point halo, (TIL_TR + 8) x (TIL_TC + 8) values of G, into shared memory
// with coalesced loads (columns wrapped mod N, rows past the half grid
// zero), forms its units' results from shared memory and stores them to the
// polar buffer F[img][j][l] (l < n_theta/2) through the block's node list.
// The CTAs of one image run together, so its grid is read from L2 about
// (1 + 8/48)^2 times instead of once per node gather.  Everything about the
// geometry (tiles, units, weights in float64, bank-slot order, node lists) is
// built by the plan on the host (ffb_tile_prepare).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "ffb_internal.cuh"

#define TIL_NT 256                 // threads per CTA
#define TIL_GU TIL_NT              // units per block: one per thread
#define TIL_NU 4                   // nodes per unit (at most)
#define TIL_UW 9                   // union side: W + 1
#define TIL_REC 19                 // float4 planes of a unit record: 9 column, 9 row, 1 meta
#define TIL_TR 48                  // window-origin rows of a tile
#define TIL_TC 48                  // window-origin columns of a tile
#define TIL_RS (TIL_TR + 8)        // rows of the tile in shared memory (origins + the union's reach)
#define TIL_CS (TIL_TC + 8)        // columns of the tile in shared memory
#define TIL_CP (TIL_CS + 1)        // row pitch (odd: rows start in different banks)

// ---------------------------------------------------------------------------
// One CTA per (block, image).  block = (first G row e0, first unwrapped
// column u0, first entry of its node list, node count).  Unit record s of the
// block holds, as TIL_REC planes of TIL_GU float4 (the layout of ffb_grid.cu):
//   plane q      (q < 9)  the column weights of union column q per node slot
//   plane 9 + r  (r < 9)  the row weights of union row r per node slot
//   plane 18              (ru | cu << 16, slot0 | slot1 << 16,
//                          slot2 | slot3 << 16, 0): union origin in the tile
//                          and the node slots (indices into the block's node
//                          list; 0xFFFF: none, zero weights)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TIL_NT, 3)
k_interp_tile(const float2 *__restrict__ G, int N, int h, int Mh, int nh, int n_xi,
              const float4 *__restrict__ units, const int4 *__restrict__ blocks, const int *__restrict__ nodes,
              float2 *__restrict__ F, int *status) {
    __shared__ float2 T[TIL_RS * TIL_CP];
    __shared__ float2 stage[TIL_NU * TIL_GU];
    const int4 blk = __ldg(&blocks[blockIdx.x]);
    const int e0 = blk.x, u0 = blk.y, nb0 = blk.z, cnt = blk.w;
    const int img = blockIdx.y;
    const float2 *Gi = G + (size_t)img * Mh * N;
    // the tile: row i is G row e0 + i (zero past the half grid), column c is
    // m1 = u0 + c - N/2 - h, stored at m1 mod N
    for (int i = threadIdx.x; i < TIL_RS * TIL_CS; i += TIL_NT) {
        const int r = i / TIL_CS, c = i - r * TIL_CS;
        const int e = e0 + r;
        int col = (u0 + c - N / 2 - h) % N;
        if (col < 0) col += N;
        T[r * TIL_CP + c] = (e < Mh) ? __ldg(&Gi[(size_t)e * N + col]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int s = threadIdx.x;
    const float4 *rec = units + (size_t)blockIdx.x * TIL_REC * TIL_GU;
    const float4 meta = __ldg(&rec[18 * TIL_GU + s]);
    const unsigned s01 = __float_as_uint(meta.y), s23 = __float_as_uint(meta.z);
    const int sl[4] = {(int)(s01 & 0xFFFFu), (int)(s01 >> 16), (int)(s23 & 0xFFFFu), (int)(s23 >> 16)};
    if (sl[0] < cnt) {
        const int rc = __float_as_int(meta.x);
        const int r0 = rc & 0xFFFF, c0 = rc >> 16;
        float2 acc[TIL_NU];
#pragma unroll
        for (int n = 0; n < TIL_NU; ++n) acc[n] = make_float2(0.f, 0.f);
        if (r0 + TIL_UW > TIL_RS || c0 + TIL_UW > TIL_CS) {
            ffb_flag(status, FFB_ERR_ARG);
        } else {
            float wx[TIL_UW][TIL_NU];
#pragma unroll
            for (int q = 0; q < TIL_UW; ++q) {
                const float4 v = __ldg(&rec[q * TIL_GU + s]);
                wx[q][0] = v.x;
                wx[q][1] = v.y;
                wx[q][2] = v.z;
                wx[q][3] = v.w;
            }
            // row by row: the union row interpolated with each node's column
            // weights, then weighted by the node's row weight
            const float2 *base = T + r0 * TIL_CP + c0;
#pragma unroll 1
            for (int r = 0; r < TIL_UW; ++r) {
                const float4 wv = __ldg(&rec[(TIL_UW + r) * TIL_GU + s]);
                const float wy[4] = {wv.x, wv.y, wv.z, wv.w};
                const float2 *row = base + r * TIL_CP;
                float2 u[TIL_NU];
#pragma unroll
                for (int n = 0; n < TIL_NU; ++n) u[n] = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < TIL_UW; ++q) {
                    const float2 g = row[q];
#pragma unroll
                    for (int n = 0; n < TIL_NU; ++n) {
                        u[n].x = fmaf(wx[q][n], g.x, u[n].x);
                        u[n].y = fmaf(wx[q][n], g.y, u[n].y);
                    }
                }
#pragma unroll
                for (int n = 0; n < TIL_NU; ++n) {
                    acc[n].x = fmaf(wy[n], u[n].x, acc[n].x);
                    acc[n].y = fmaf(wy[n], u[n].y, acc[n].y);
                }
            }
        }
#pragma unroll
        for (int n = 0; n < TIL_NU; ++n)
            if (sl[n] < cnt) stage[sl[n]] = acc[n];
    }
    __syncthreads();
    // results in the order of the block's node list (node t = j nh + l)
    float2 *Fi = F + (size_t)img * n_xi * nh;
    for (int i = threadIdx.x; i < cnt; i += TIL_NT) Fi[__ldg(&nodes[nb0 + i])] = stage[i];
}

// ---------------------------------------------------------------------------
// Adjoint of k_interp_tile (step a10): the polar values g (inverse ring DFT,
// layout of the polar buffer) spread into the block's tile in shared memory,
// T[ru + r][cu + q] += sum_n wy_n[r] wx_n[q] g_n over a unit's nodes (one
// shared-memory atomic per value of the 9 x 9 union and component), then the
// tile added into the half grid Gext (zeroed by the caller) at G row e0 + r,
// column (u0 + c - N/2 - h) mod N with global atomics (tiles overlap in their
// halos, and a tile may have several blocks); cells no unit touched are
// skipped.  The transpose of the forward with the same weights, so the
// adjoint stays exact against it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TIL_NT, 3)
k_adj_spread_tile(const float2 *__restrict__ Gpol, int N, int h, int Mh, int nh, int n_xi,
                  const float4 *__restrict__ units, const int4 *__restrict__ blocks, const int *__restrict__ nodes,
                  float2 *__restrict__ Gext, int *status) {
    __shared__ float2 T[TIL_RS * TIL_CP];
    float *Tf = (float *)T;
    for (int i = threadIdx.x; i < TIL_RS * TIL_CP; i += TIL_NT) T[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int4 blk = __ldg(&blocks[blockIdx.x]);
    const int e0 = blk.x, u0 = blk.y, nb0 = blk.z, cnt = blk.w;
    const int img = blockIdx.y;
    const float2 *Gp = Gpol + (size_t)img * n_xi * nh;
    const int s = threadIdx.x;
    const float4 *rec = units + (size_t)blockIdx.x * TIL_REC * TIL_GU;
    const float4 meta = __ldg(&rec[18 * TIL_GU + s]);
    const unsigned s01 = __float_as_uint(meta.y), s23 = __float_as_uint(meta.z);
    const int sl[4] = {(int)(s01 & 0xFFFFu), (int)(s01 >> 16), (int)(s23 & 0xFFFFu), (int)(s23 >> 16)};
    if (sl[0] < cnt) {
        const int rc = __float_as_int(meta.x);
        const int r0 = rc & 0xFFFF, c0 = rc >> 16;
        if (r0 + TIL_UW > TIL_RS || c0 + TIL_UW > TIL_CS) {
            ffb_flag(status, FFB_ERR_ARG);
        } else {
            float2 v[TIL_NU];
#pragma unroll
            for (int n = 0; n < TIL_NU; ++n)
                v[n] = (sl[n] < cnt) ? __ldg(&Gp[__ldg(&nodes[nb0 + sl[n]])]) : make_float2(0.f, 0.f);
            float4 wx[TIL_UW];
#pragma unroll
            for (int q = 0; q < TIL_UW; ++q) wx[q] = __ldg(&rec[q * TIL_GU + s]);
            float *base = Tf + 2 * (r0 * TIL_CP + c0);
#pragma unroll 1
            for (int r = 0; r < TIL_UW; ++r) {
                const float4 wy = __ldg(&rec[(TIL_UW + r) * TIL_GU + s]);
                const float2 a0 = make_float2(wy.x * v[0].x, wy.x * v[0].y), a1 = make_float2(wy.y * v[1].x, wy.y * v[1].y);
                const float2 a2 = make_float2(wy.z * v[2].x, wy.z * v[2].y), a3 = make_float2(wy.w * v[3].x, wy.w * v[3].y);
                float *row = base + 2 * r * TIL_CP;
#pragma unroll
                for (int q = 0; q < TIL_UW; ++q) {
                    const float re = fmaf(wx[q].x, a0.x, fmaf(wx[q].y, a1.x, fmaf(wx[q].z, a2.x, wx[q].w * a3.x)));
                    const float im = fmaf(wx[q].x, a0.y, fmaf(wx[q].y, a1.y, fmaf(wx[q].z, a2.y, wx[q].w * a3.y)));
                    atomicAdd(&row[2 * q], re);
                    atomicAdd(&row[2 * q + 1], im);
                }
            }
        }
    }
    __syncthreads();
    float2 *Gi = Gext + (size_t)img * Mh * N;
    for (int i = threadIdx.x; i < TIL_RS * TIL_CS; i += TIL_NT) {
        const int r = i / TIL_CS, c = i - r * TIL_CS;
        const int e = e0 + r;
        const float2 val = T[r * TIL_CP + c];
        if (e >= Mh || (val.x == 0.f && val.y == 0.f)) continue;
        int col = (u0 + c - N / 2 - h) % N;
        if (col < 0) col += N;
        atomicAdd(&Gi[(size_t)e * N + col], val);
    }
}

// ---------------------------------------------------------------------------
// The tile table (host, float64).  Node t = j nh + l, l < nh = n_theta/2,
// sits at p = N xi_j (cos theta_l, sin theta_l) in grid units; its window
// starts at m = ceil(p - W/2) with weights phi(f - b), f = p - m, b = 0..7,
// phi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) (the ES kernel of the plan).
// Within a tile the nodes are sorted by origin and grouped: the first node
// not yet taken anchors a unit and takes up to three more untaken nodes
// whose origins lie in the 2 x 2 box from its own, same origin first, then
// right, below, below right.  A tile's units go to blocks of at most TIL_GU
// in that order; within a block the units are ordered per half warp with
// distinct bank slots (union origin ru TIL_CP + cu) mod 16, a unit whose
// nodes all sit in the union's first row (column) starting one row (column)
// earlier where that evens out the slots.
// ---------------------------------------------------------------------------
static int build_tiles(int N, int W, double beta, int n_xi, int n_theta, const double *xi,
                       std::vector<float4> &rec, std::vector<int4> &blk, std::vector<int> &nodes) {
    if (W != 8 || N < 16 || n_xi < 1 || n_theta < 4 || (n_theta & 1) || !xi) return FFB_ERR_UNSUPPORTED;
    const int h = (W + 1) / 2, Mh = N / 2 + 1 + 2 * h, nh = n_theta / 2;
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
        int t, r0, u;   // node index, window origin (G row, unwrapped column)
        double f1, f2;
    };
    // nodes per tile, keyed (tile row, tile column)
    std::map<std::pair<int, int>, std::vector<Node>> tiles;
    for (int j = 0; j < n_xi; ++j)
        for (int l = 0; l < nh; ++l) {
            const double th = 2.0 * M_PI * (double)l / (double)n_theta;
            const double p1 = N * xi[j] * std::cos(th), p2 = N * xi[j] * std::sin(th);
            const double m1 = std::ceil(p1 - 0.5 * W), m2 = std::ceil(p2 - 0.5 * W);
            const int r0 = (int)m2 + h, u = (int)m1 + N / 2 + h;
            if (r0 < 0 || r0 + W > Mh || u < 0 || u + W > N + 2 * h) return FFB_ERR_UNSUPPORTED;
            tiles[{r0 / TIL_TR, u / TIL_TC}].push_back({j * nh + l, r0, u, p1 - m1, p2 - m2});
        }
    rec.clear();
    blk.clear();
    nodes.clear();
    for (auto &kv : tiles) {
        const int e0 = kv.first.first * TIL_TR, u0 = kv.first.second * TIL_TC;
        std::vector<Node> &nd = kv.second;
        std::stable_sort(nd.begin(), nd.end(), [](const Node &a, const Node &b) {
            return (a.r0 != b.r0) ? a.r0 < b.r0 : a.u < b.u;
        });
        // units: indices into nd
        std::map<std::pair<int, int>, std::vector<int>> at;   // origin -> untaken nodes
        for (int i = 0; i < (int)nd.size(); ++i) at[{nd[i].r0, nd[i].u}].push_back(i);
        std::vector<char> used(nd.size(), 0);
        std::vector<std::vector<int>> un;
        for (int i = 0; i < (int)nd.size(); ++i) {
            if (used[i]) continue;
            std::vector<int> u{i};
            used[i] = 1;
            const int r = nd[i].r0, c = nd[i].u;
            const int cells[4][2] = {{r, c}, {r, c + 1}, {r + 1, c}, {r + 1, c + 1}};
            for (int cc = 0; cc < 4 && (int)u.size() < TIL_NU; ++cc) {
                auto it = at.find({cells[cc][0], cells[cc][1]});
                if (it == at.end()) continue;
                for (int k : it->second)
                    if (!used[k] && (int)u.size() < TIL_NU) {
                        used[k] = 1;
                        u.push_back(k);
                    }
            }
            un.push_back(u);
        }
        for (size_t b0 = 0; b0 < un.size(); b0 += TIL_GU) {
            const int nu = (int)std::min<size_t>(TIL_GU, un.size() - b0);
            const int list0 = (int)nodes.size();
            // union origins in tile coordinates, balanced over the bank slots
            std::vector<int> urow(nu), ucol(nu);
            std::vector<std::vector<std::pair<int, int>>> cand(nu);
            int cnt16[16] = {};
            for (int a = 0; a < nu; ++a) {
                int rmin = 1 << 30, rmax = -1, cmin = 1 << 30, cmax = -1;
                for (int k : un[b0 + a]) {
                    rmin = std::min(rmin, nd[k].r0 - e0);
                    rmax = std::max(rmax, nd[k].r0 - e0);
                    cmin = std::min(cmin, nd[k].u - u0);
                    cmax = std::max(cmax, nd[k].u - u0);
                }
                const bool mr = (rmax == rmin) && rmin >= 1, mc = (cmax == cmin) && cmin >= 1;
                cand[a].push_back({rmin, cmin});
                if (mc) cand[a].push_back({rmin, cmin - 1});
                if (mr) cand[a].push_back({rmin - 1, cmin});
                if (mr && mc) cand[a].push_back({rmin - 1, cmin - 1});
                urow[a] = rmin;
                ucol[a] = cmin;
                if (cand[a].size() == 1) cnt16[(rmin * TIL_CP + cmin) & 15]++;
            }
            for (int a = 0; a < nu; ++a) {
                if (cand[a].size() == 1) continue;
                int best = 0;
                for (int k = 1; k < (int)cand[a].size(); ++k)
                    if (cnt16[(cand[a][k].first * TIL_CP + cand[a][k].second) & 15] <
                        cnt16[(cand[a][best].first * TIL_CP + cand[a][best].second) & 15])
                        best = k;
                urow[a] = cand[a][best].first;
                ucol[a] = cand[a][best].second;
                cnt16[(urow[a] * TIL_CP + ucol[a]) & 15]++;
            }
            std::vector<int> bucket[16];
            for (int a = nu - 1; a >= 0; --a) bucket[(urow[a] * TIL_CP + ucol[a]) & 15].push_back(a);
            const size_t base = rec.size();
            rec.resize(base + (size_t)TIL_REC * TIL_GU, make_float4(0.f, 0.f, 0.f, 0.f));
            float4 *R = rec.data() + base;
            for (int s = 0; s < TIL_GU; ++s) R[18 * TIL_GU + s] = make_float4(0.f, bits(0xFFFFFFFFu), bits(0xFFFFFFFFu), 0.f);
            int pos = 0;
            auto put = [&](int a) {
                const int ru = urow[a], cu = ucol[a];
                if (ru < 0 || cu < 0 || ru + TIL_UW > TIL_RS || cu + TIL_UW > TIL_CS) return false;
                float wx[TIL_UW][4] = {}, wy[TIL_UW][4] = {};
                unsigned slot[4] = {0xFFFFu, 0xFFFFu, 0xFFFFu, 0xFFFFu};
                int i = 0;
                for (int k : un[b0 + a]) {
                    const Node &v = nd[k];
                    const int dr = v.r0 - e0 - ru, dc = v.u - u0 - cu;   // 0 or 1
                    for (int q = 0; q < W; ++q) {
                        wx[dc + q][i] = (float)phi(v.f1 - q);
                        wy[dr + q][i] = (float)phi(v.f2 - q);
                    }
                    slot[i] = (unsigned)((int)nodes.size() - list0);
                    nodes.push_back(v.t);
                    ++i;
                }
                for (int q = 0; q < TIL_UW; ++q) {
                    R[q * TIL_GU + pos] = make_float4(wx[q][0], wx[q][1], wx[q][2], wx[q][3]);
                    R[(TIL_UW + q) * TIL_GU + pos] = make_float4(wy[q][0], wy[q][1], wy[q][2], wy[q][3]);
                }
                R[18 * TIL_GU + pos] = make_float4(bits((unsigned)ru | ((unsigned)cu << 16)),
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
            blk.push_back(make_int4(e0, u0, list0, (int)nodes.size() - list0));
        }
    }
    return FFB_OK;
}

// the plan's tile table (separate-kernel plans with w = 8)
int ffb_tile_prepare(ffb_plan_t p, cudaStream_t s) {
    if (p->w != 8 || p->fused) return FFB_OK;   // the per-node kernel stays in use
    std::vector<double> xi(p->n_xi);
    int e = ffb_check_cuda(cudaMemcpyAsync(xi.data(), p->d_xi, sizeof(double) * p->n_xi, cudaMemcpyDeviceToHost, s));
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (e) return e;
    std::vector<float4> rec;
    std::vector<int4> blk;
    std::vector<int> nodes;
    if ((e = build_tiles(p->N, p->w, p->beta, p->n_xi, p->n_theta, xi.data(), rec, blk, nodes))) return e;
    e = ffb_check_cuda(cudaMalloc((void **)&p->d_tunits, sizeof(float4) * rec.size()));
    if (!e) e = ffb_check_cuda(cudaMalloc((void **)&p->d_tblk, sizeof(int4) * blk.size()));
    if (!e) e = ffb_check_cuda(cudaMalloc((void **)&p->d_tnodes, sizeof(int) * nodes.size()));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_tunits, rec.data(), sizeof(float4) * rec.size(),
                                               cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_tblk, blk.data(), sizeof(int4) * blk.size(),
                                               cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaMemcpyAsync(p->d_tnodes, nodes.data(), sizeof(int) * nodes.size(),
                                               cudaMemcpyHostToDevice, s));
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (!e) p->ntblk = (int)blk.size();
    return e;
}

// a3 for nimg images of the chunk: the half grids p->d_G -> polar samples F
int ffb_launch_tile_polar(ffb_plan_t p, int nimg, float2 *F, cudaStream_t s) {
    if (p->ntblk <= 0) return FFB_ERR_STATE;
    dim3 g(p->ntblk, nimg);
    ProfScope ps(p, FFB_KC_INTERP, s);
    k_interp_tile<<<g, TIL_NT, 0, s>>>(p->d_G, p->N, p->h, p->Mh, p->n_theta / 2, p->n_xi, p->d_tunits, p->d_tblk,
                                       p->d_tnodes, F, p->d_status);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

// the adjoint's spreading for nimg images: polar values Gpol -> Gext (zeroed)
int ffb_launch_tile_spread(ffb_plan_t p, int nimg, const float2 *Gpol, float2 *Gext, cudaStream_t s) {
    if (p->ntblk <= 0) return FFB_ERR_STATE;
    dim3 g(p->ntblk, nimg);
    ProfScope ps(p, FFB_KC_ADJ_SPREAD, s);
    k_adj_spread_tile<<<g, TIL_NT, 0, s>>>(Gpol, p->N, p->h, p->Mh, p->n_theta / 2, p->n_xi, p->d_tunits, p->d_tblk,
                                           p->d_tnodes, Gext, p->d_status);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}

extern "C" int ffb_tile_units(int N, int w, double beta, int n_xi, int n_theta, const double *h_xi,
                              int64_t *h_counts, float *h_rec, int *h_blk, int *h_nodes) {
    if (!h_counts || !h_xi || n_xi < 1 || n_theta < 4 || !(beta > 0.0)) return FFB_ERR_ARG;
    std::vector<float4> rec;
    std::vector<int4> blk;
    std::vector<int> nodes;
    const int e = build_tiles(N, w, beta, n_xi, n_theta, h_xi, rec, blk, nodes);
    if (e) return e;
    h_counts[0] = (int64_t)blk.size();
    h_counts[1] = (int64_t)nodes.size();
    h_counts[2] = TIL_REC;
    h_counts[3] = TIL_GU;
    h_counts[4] = TIL_TR;
    h_counts[5] = TIL_TC;
    h_counts[6] = TIL_RS;
    h_counts[7] = TIL_CS;
    h_counts[8] = TIL_CP;
    if (h_rec) std::memcpy(h_rec, rec.data(), sizeof(float4) * rec.size());
    if (h_blk) std::memcpy(h_blk, blk.data(), sizeof(int4) * blk.size());
    if (h_nodes) std::memcpy(h_nodes, nodes.data(), sizeof(int) * nodes.size());
    return FFB_OK;
}
