// ffb_group.cu -- many stacks of uneven L and n in one call (batching).
//
// Sec. IV observes that the expansion and the covariance are sums over
// images that split freely among workers.  A group holds S independent stacks,
// each with its own plan (its own L, c, R, tables and covariance), and runs
// a1-a7 for all of them in one call:
//   * every stack's expansion (a1-a5: grid, interpolation, ring FFT, radial
//     quadrature, chunk by chunk) runs on its own branch stream, so stacks too
//     small to fill the GPU overlap;
//   * the covariance of all stacks (a6/a7) is one persistent launch over a
//     stack table of (stack, k block or FP32 tile, image range) items: a
//     grouped SYRK over the uneven per-k block sizes p_k of every stack
//     (k_tc_cov / k_cov_fp32 with a CovGroup of S stacks);
//   * the launches of one call form a CUDA graph: the first call with a given
//     set of pointers, sizes and reset flags runs eagerly (and, once per group,
//     times the candidate item shapes of the grouped launch: the autotuner);
//     the second captures the same launches into a graph; later calls replay it.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ffb_internal.cuh"

#define CKG(call)                    \
    do {                             \
        int _s = (call);             \
        if (_s != FFB_OK) return _s; \
    } while (0)

namespace {

struct Key {
    int mode;                           // 1: expand + covariance, 2: covariance only
    std::vector<const void *> images, coef;
    std::vector<int64_t> n;
    std::vector<char> reset;            // per stack: accumulator restarted in this call
    bool operator==(const Key &o) const {
        return mode == o.mode && images == o.images && coef == o.coef && n == o.n && reset == o.reset;
    }
};

struct Round {
    int S = 0;                          // stacks with images in this round
    int nitems = 0;                     // (stack, k, M tile) items of the grouped quadrature
    size_t first = 0;                   // index of the round's first stack descriptor
};

struct Entry {
    Key key;
    int seen = 0;                       // calls so far with this key
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> plan_launches; // kernel launches per call, per plan
    int64_t group_launches = 0;         // the grouped launches per call
    std::vector<Round> rounds;          // grouped quadrature rounds (tensor-core groups)
    void *d_desc = nullptr;             // their stack descriptors, device memory
};

struct Cand {
    int per, tile, grid;
    float ms;
};

}  // namespace

struct ffb_group_s {
    int S = 0;
    int precision = 0;
    std::vector<ffb_plan_t> plans;
    cudaStream_t cap = nullptr;          // capture stream
    std::vector<cudaStream_t> br;        // one branch stream per stack
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    int *d_status = nullptr;             // status word of the grouped launches
    double *d_scratch = nullptr;         // tuner's accumulator (results discarded)
    size_t scratch_len = 0;
    // autotuner
    int tuned = 0, per = 0, tile = 32, grid = 0;
    std::vector<Cand> cands;
    // grouped quadrature: widest block of the members, launch shape (CTAs per
    // SM, pipeline stages) chosen by the tuner, and its timings
    int BNmax = 0, q_tuned = 0, q_per_sm = 1, q_nst = 0;
    std::vector<Cand> qcands;           // per = CTAs per SM, tile = stages
    // graph cache
    std::vector<Entry> cache;
    int64_t graphs = 0, replays = 0, eager = 0, last_launches = 0;
};

static void drop_entry(Entry &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.d_desc) cudaFree(e.d_desc);
    e.exec = nullptr;
    e.d_desc = nullptr;
}

static void release(ffb_group_t g) {
    for (Entry &e : g->cache) drop_entry(e);
    for (cudaStream_t s : g->br)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->join)
        if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->d_status) cudaFree(g->d_status);
    if (g->d_scratch) cudaFree(g->d_scratch);
    delete g;
}

extern "C" int ffb_group_create(ffb_group_t *out, int S, const ffb_plan_t *plans, void *stream) {
    if (!out || !plans || S < 1 || S > FFB_GROUP_MAX) return FFB_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < S; ++i) {
        FFB_PLAN_HERE(plans[i]);   // every member lives on the current device
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return FFB_ERR_ARG;   // a plan's scratch serves one stack
        if (plans[i]->precision != plans[0]->precision) return FFB_ERR_ARG;
    }
    const int prec = plans[0]->precision;
    for (int i = 0; i < S; ++i)
        if (prec != FFB_FP32 && !ffb_tc_cov_supported(plans[i])) return FFB_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    ffb_group_t g = new ffb_group_s();
    g->S = S;
    g->precision = prec;
    g->plans.assign(plans, plans + S);
    g->br.assign(S, nullptr);
    g->join.assign(S, nullptr);
    int e = FFB_OK;
    // everything a captured launch needs exists before the first capture
    for (int i = 0; i < S && !e; ++i) {
        e = ffb_ensure_scratch(plans[i]);
        if (!e && prec != FFB_FP32) e = ffb_tc_prepare(plans[i], s, nullptr);
        if (!e) e = ffb_check_cuda(cudaStreamCreateWithFlags(&g->br[i], cudaStreamNonBlocking));
        if (!e) e = ffb_check_cuda(cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming));
    }
    if (!e) e = ffb_check_cuda(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
    if (!e) e = ffb_check_cuda(cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
    if (!e) e = ffb_check_cuda(cudaMalloc(&g->d_status, sizeof(int)));
    if (!e) e = ffb_check_cuda(cudaMemsetAsync(g->d_status, 0, sizeof(int), s));
    if (!e) {
        size_t len = 0;
        for (ffb_plan_t p : g->plans) len = std::max(len, (size_t)p->cov_total + p->p[0]);
        g->scratch_len = len;
        e = ffb_check_cuda(cudaMalloc(&g->d_scratch, sizeof(double) * len));
    }
    if (!e && prec != FFB_FP32) {
        for (ffb_plan_t p : g->plans) g->BNmax = std::max(g->BNmax, ffb_tc_bn(p));
        int per_sm[4], nst[4];
        if (ffb_tc_group_shapes(prec, g->BNmax, per_sm, nst) <= 0) e = FFB_ERR_UNSUPPORTED;
        else {
            g->q_per_sm = per_sm[0];
            g->q_nst = nst[0];
        }
    }
    if (!e) e = ffb_check_cuda(cudaStreamSynchronize(s));
    if (e) {
        release(g);
        return e;
    }
    *out = g;
    return FFB_OK;
}

extern "C" int ffb_group_destroy(ffb_group_t g) {
    if (!g) return FFB_OK;
    cudaDeviceSynchronize();
    release(g);
    return FFB_OK;
}

// stack table of the grouped covariance for the stacks with images
static void build_table(ffb_group_t g, const Key &k, int per, int tile, bool scratch, CovGroup *cg) {
    const bool tc = g->precision != FFB_FP32;
    cg->S = 0;
    cg->tile_imgs = tile;
    cg->nitems = 0;
    for (int i = 0; i < g->S; ++i) {
        if (k.n[i] <= 0) continue;
        CovStack &st = cg->st[cg->S++];
        ffb_cov_stack(g->plans[i], (const float *)k.coef[i], k.n[i], tc, &st);
        st.per = per;
        st.item0 = cg->nitems;
        if (scratch) {
            st.acc = g->d_scratch;
            st.sum0 = g->d_scratch + (g->scratch_len - g->plans[i]->p[0]);
        }
        cg->nitems += (int64_t)st.nk * ((k.n[i] + per - 1) / per);
    }
}

// times the candidate item shapes of the grouped covariance on this call's
// coefficients, accumulating into scratch; keeps the fastest
static int tune(ffb_group_t g, const Key &k, cudaStream_t s) {
    const bool tc = g->precision != FFB_FP32;
    std::vector<Cand> cands;
    const int grid0 = ffb_cov_grid_default(g->precision);
    if (tc) {
        for (int per : {128, 256, 512}) cands.push_back({per, 32, grid0, 0.f});
    } else {
        for (int per : {512, 1024, 2048, 4096})
            for (int gm : {1, 2}) cands.push_back({per, 32, grid0 * gm, 0.f});
    }
    cudaEvent_t a, b;
    CKG(ffb_check_cuda(cudaEventCreate(&a)));
    CKG(ffb_check_cuda(cudaEventCreate(&b)));
    int e = FFB_OK;
    CovGroup cg;
    for (size_t c = 0; c <= cands.size() && !e; ++c) {
        const Cand &cd = cands[c == 0 ? 0 : c - 1];   // the first candidate runs twice (warm-up)
        build_table(g, k, cd.per, cd.tile, true, &cg);
        e = ffb_check_cuda(cudaEventRecord(a, s));
        if (!e) e = ffb_launch_cov_group(g->precision, cg, cd.grid, g->d_status, s);
        if (!e) e = ffb_check_cuda(cudaEventRecord(b, s));
        if (!e) e = ffb_check_cuda(cudaEventSynchronize(b));
        float ms = 0.f;
        if (!e) e = ffb_check_cuda(cudaEventElapsedTime(&ms, a, b));
        if (c > 0) cands[c - 1].ms = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e) return e;
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (cands[c].ms < cands[best].ms) best = c;
    g->per = cands[best].per;
    g->tile = cands[best].tile;
    g->grid = cands[best].grid;
    g->cands = cands;
    g->tuned = 1;
    return FFB_OK;
}

// images per round of stack i: one group of chunks of its plan
static int64_t round_images(ffb_plan_t p) { return (int64_t)ffb_tc_group(p) * p->chunk; }

// the rounds of a tensor-core group call: round r holds the r-th group of
// chunks of every stack that has one, its stacks' descriptors packed with
// rising item numbers; built once per call shape (outside any capture)
static int build_rounds(ffb_group_t g, const Key &k, Entry *ent) {
    const size_t sb = ffb_tc_stack_bytes();
    std::vector<unsigned char> host;
    int nr = 0;
    for (int i = 0; i < g->S; ++i)
        if (k.n[i] > 0) nr = std::max<int64_t>(nr, (k.n[i] + round_images(g->plans[i]) - 1) / round_images(g->plans[i]));
    ent->rounds.assign(nr, Round());
    for (int r = 0; r < nr; ++r) {
        Round &R = ent->rounds[r];
        R.first = host.size() / sb;
        for (int i = 0; i < g->S; ++i) {
            ffb_plan_t p = g->plans[i];
            const int64_t per = round_images(p), g0 = (int64_t)r * per;
            if (k.n[i] <= g0) continue;
            const int64_t g1 = std::min<int64_t>(k.n[i], g0 + per);
            host.resize(host.size() + sb);
            int items = 0;
            CKG(ffb_tc_stack_fill(p, (float *)k.coef[i] + (size_t)g0 * p->P * 2, (int)(g1 - g0), R.nitems,
                                  host.data() + host.size() - sb, &items));
            R.nitems += items;
            R.S++;
        }
    }
    if (host.empty()) return FFB_OK;
    CKG(ffb_check_cuda(cudaMalloc(&ent->d_desc, host.size())));
    return ffb_check_cuda(cudaMemcpy(ent->d_desc, host.data(), host.size(), cudaMemcpyHostToDevice));
}

static int quad_launch(ffb_group_t g, const Entry *ent, int r, int per_sm, int nst, cudaStream_t s) {
    const Round &R = ent->rounds[r];
    const char *d = (const char *)ent->d_desc + R.first * ffb_tc_stack_bytes();
    return ffb_tc_group_bessel(g->precision, d, R.S, R.nitems, g->BNmax, per_sm, nst, g->d_status,
                               g->plans[0]->wait_budget, s);
}

// times the launch shapes of the grouped quadrature on round r of this call
// (its operands are ready; every run writes the same coefficients) and keeps
// the fastest
static int tune_quad(ffb_group_t g, const Entry *ent, int r, cudaStream_t s) {
    int per_sm[4], nst[4];
    const int nc = ffb_tc_group_shapes(g->precision, g->BNmax, per_sm, nst);
    cudaEvent_t a, b;
    CKG(ffb_check_cuda(cudaEventCreate(&a)));
    CKG(ffb_check_cuda(cudaEventCreate(&b)));
    std::vector<Cand> cands;
    for (int c = 0; c < nc; ++c) cands.push_back({per_sm[c], nst[c], 0, 0.f});
    int e = FFB_OK;
    for (int c = 0; c <= nc && !e; ++c) {
        const Cand &cd = cands[c == 0 ? 0 : c - 1];   // the first shape runs twice (warm-up)
        e = ffb_check_cuda(cudaEventRecord(a, s));
        if (!e) e = quad_launch(g, ent, r, cd.per, cd.tile, s);
        if (!e) e = ffb_check_cuda(cudaEventRecord(b, s));
        if (!e) e = ffb_check_cuda(cudaEventSynchronize(b));
        float ms = 0.f;
        if (!e) e = ffb_check_cuda(cudaEventElapsedTime(&ms, a, b));
        if (c > 0) cands[c - 1].ms = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e) return e;
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (cands[c].ms < cands[best].ms) best = c;
    g->q_per_sm = cands[best].per;
    g->q_nst = cands[best].tile;
    g->qcands = cands;
    g->q_tuned = 1;
    return FFB_OK;
}

// the launches of one call on stream `main` (the user's stream, or the
// capture stream); each stack's expansion on its branch.  Tensor-core groups
// run in rounds: every stack's next group of chunks through a1-a4 on its
// branch, then one grouped quadrature launch over all of them
static int run(ffb_group_t g, const Key &k, cudaStream_t main, Entry *ent, bool count) {
    std::vector<int64_t> before(g->S);
    for (int i = 0; i < g->S; ++i) before[i] = g->plans[i]->launches;
    int64_t gl = 0;
    if (k.mode == 1 && g->precision == FFB_FP32) {
        CKG(ffb_check_cuda(cudaEventRecord(g->fork, main)));
        for (int i = 0; i < g->S; ++i) {
            if (k.n[i] <= 0) continue;
            CKG(ffb_check_cuda(cudaStreamWaitEvent(g->br[i], g->fork, 0)));
            CKG(ffb_expand_on(g->plans[i], (const float *)k.images[i], k.n[i], (float *)k.coef[i], g->br[i]));
            CKG(ffb_check_cuda(cudaEventRecord(g->join[i], g->br[i])));
            CKG(ffb_check_cuda(cudaStreamWaitEvent(main, g->join[i], 0)));
        }
    } else if (k.mode == 1) {
        for (size_t r = 0; r < ent->rounds.size(); ++r) {
            CKG(ffb_check_cuda(cudaEventRecord(g->fork, main)));
            for (int i = 0; i < g->S; ++i) {
                ffb_plan_t p = g->plans[i];
                const int64_t per = round_images(p), g0 = (int64_t)r * per;
                if (k.n[i] <= g0) continue;
                const int64_t g1 = std::min<int64_t>(k.n[i], g0 + per);
                CKG(ffb_check_cuda(cudaStreamWaitEvent(g->br[i], g->fork, 0)));
                CKG(ffb_expand_part(p, (const float *)k.images[i], g0, g1, g->br[i]));
                if (!p->ring_direct) CKG(ffb_tc_split_planes(p, g->br[i]));
                CKG(ffb_check_cuda(cudaEventRecord(g->join[i], g->br[i])));
                CKG(ffb_check_cuda(cudaStreamWaitEvent(main, g->join[i], 0)));
            }
            if (!g->q_tuned) CKG(tune_quad(g, ent, (int)r, main));
            CKG(quad_launch(g, ent, (int)r, g->q_per_sm, g->q_nst, main));
            ++gl;
        }
    }
    for (int i = 0; i < g->S; ++i) {
        if (!k.reset[i]) continue;
        ffb_plan_t p = g->plans[i];
        CKG(ffb_check_cuda(cudaMemsetAsync(p->d_acc, 0, sizeof(double) * p->cov_total, main)));
        CKG(ffb_check_cuda(cudaMemsetAsync(p->d_sum0, 0, sizeof(double) * p->p[0], main)));
        if (k.n[i] > 0) CKG(ffb_launch_cov_shift(p, (const float *)k.coef[i], k.n[i], main));
    }
    if (!g->tuned) CKG(tune(g, k, main));
    CovGroup cg;
    build_table(g, k, g->per, g->tile, false, &cg);
    if (cg.nitems > 0) {
        CKG(ffb_launch_cov_group(g->precision, cg, g->grid, g->d_status, main));
        ++gl;
    }
    if (count) {
        ent->plan_launches.resize(g->S);
        for (int i = 0; i < g->S; ++i) ent->plan_launches[i] = g->plans[i]->launches - before[i];
        ent->group_launches = gl;
    }
    return FFB_OK;
}

static int call(ffb_group_t g, Key &k, cudaStream_t s) {
    for (int i = 0; i < g->S; ++i)
        if (g->plans[i]->precision != g->precision) return FFB_ERR_STATE;   // ffb_set_precision since create
    for (int i = 0; i < g->S; ++i) {
        ffb_plan_t p = g->plans[i];
        if (k.n[i] > 0 && !p->shift_set) k.reset[i] = 1;   // the first batch fixes the pilot mean
    }
    Entry *ent = nullptr;
    for (Entry &e : g->cache)
        if (e.key == k) ent = &e;
    if (!ent) {
        if (g->cache.size() >= 8) {   // keep the cache small: drop the oldest
            drop_entry(g->cache.front());
            g->cache.erase(g->cache.begin());
        }
        g->cache.push_back(Entry());
        ent = &g->cache.back();
        ent->key = k;
        // the grouped quadrature's rounds and descriptors (allocated here,
        // never inside a capture)
        if (k.mode == 1 && g->precision != FFB_FP32) CKG(build_rounds(g, k, ent));
    }
    int e = FFB_OK;
    if (ent->seen == 0) {
        // first call with this key: eager (sets kernel attributes, tunes once)
        e = run(g, k, s, ent, true);
        g->eager++;
    } else {
        if (!ent->exec) {
            std::vector<int> prof(g->S);
            for (int i = 0; i < g->S; ++i) {
                prof[i] = g->plans[i]->prof_on;
                g->plans[i]->prof_on = 0;   // no profiling events inside a graph
            }
            std::vector<int64_t> before(g->S);
            for (int i = 0; i < g->S; ++i) before[i] = g->plans[i]->launches;
            cudaGraph_t graph = nullptr;
            e = ffb_check_cuda(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
            if (!e) {
                const int er = run(g, k, g->cap, ent, false);
                const int ee = ffb_check_cuda(cudaStreamEndCapture(g->cap, &graph));
                e = er ? er : ee;
            }
            for (int i = 0; i < g->S; ++i) {
                g->plans[i]->prof_on = prof[i];
                g->plans[i]->launches = before[i];   // counted per replay below
            }
            if (!e) e = ffb_check_cuda(cudaGraphInstantiate(&ent->exec, graph, 0));
            if (graph) cudaGraphDestroy(graph);
            if (!e) g->graphs++;
        }
        if (!e) e = ffb_check_cuda(cudaGraphLaunch(ent->exec, s));
        if (!e) {
            g->replays++;
            for (int i = 0; i < g->S; ++i) g->plans[i]->launches += ent->plan_launches[i];
        }
    }
    if (e) return e;
    ent->seen++;
    int64_t tot = ent->group_launches;
    for (int64_t v : ent->plan_launches) tot += v;
    g->last_launches = tot;
    for (int i = 0; i < g->S; ++i) {
        ffb_plan_t p = g->plans[i];
        if (k.reset[i]) {
            p->n_acc = 0;
            p->shift_set = 0;
        }
        if (k.n[i] > 0) {
            p->n_acc += k.n[i];
            p->shift_set = 1;
        }
    }
    return FFB_OK;
}

static int make_key(ffb_group_t g, int mode, const float *const *images, const int64_t *n,
                    float *const *coef, int reset, Key *k) {
    if (!g || !n || !coef || (mode == 1 && !images)) return FFB_ERR_ARG;
    k->mode = mode;
    k->images.assign(g->S, nullptr);
    k->coef.assign(g->S, nullptr);
    k->n.assign(n, n + g->S);
    k->reset.assign(g->S, (char)(reset ? 1 : 0));
    for (int i = 0; i < g->S; ++i) {
        if (n[i] < 0) return FFB_ERR_ARG;
        if (n[i] > 0 && (!coef[i] || (mode == 1 && !images[i]))) return FFB_ERR_ARG;
        k->coef[i] = coef[i];
        if (mode == 1) k->images[i] = images[i];
    }
    return FFB_OK;
}

extern "C" int ffb_group_expand_cov(ffb_group_t g, const float *const *h_images, const int64_t *h_n,
                                    float *const *h_coef, int reset, void *stream) {
    if (!g) return FFB_ERR_ARG;
    FFB_PLAN_HERE(g->plans[0]);
    Key k;
    CKG(make_key(g, 1, h_images, h_n, h_coef, reset, &k));
    return call(g, k, (cudaStream_t)stream);
}

extern "C" int ffb_group_covariance(ffb_group_t g, const float *const *h_coef, const int64_t *h_n, int reset,
                                    void *stream) {
    if (!g) return FFB_ERR_ARG;
    FFB_PLAN_HERE(g->plans[0]);
    Key k;
    CKG(make_key(g, 2, nullptr, h_n, const_cast<float *const *>(h_coef), reset, &k));
    return call(g, k, (cudaStream_t)stream);
}

extern "C" int ffb_group_sync(ffb_group_t g, void *stream) {
    if (!g) return FFB_ERR_ARG;
    FFB_PLAN_HERE(g->plans[0]);
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    CKG(ffb_check_cuda(cudaMemcpyAsync(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)));
    CKG(ffb_check_cuda(cudaStreamSynchronize(s)));
    if (st != 0) {
        cudaMemsetAsync(g->d_status, 0, sizeof(int), s);
        return st;
    }
    for (ffb_plan_t p : g->plans) CKG(ffb_sync(p, stream));
    return FFB_OK;
}

extern "C" int ffb_group_info(ffb_group_t g, int64_t *h_info) {
    if (!g || !h_info) return FFB_ERR_ARG;
    h_info[0] = g->S;
    h_info[1] = g->precision;
    h_info[2] = g->per;
    h_info[3] = g->tile;
    h_info[4] = g->grid;
    h_info[5] = g->graphs;
    h_info[6] = g->replays;
    h_info[7] = g->eager;
    h_info[8] = g->last_launches;
    h_info[9] = (int64_t)g->cands.size();
    h_info[10] = g->q_per_sm;
    h_info[11] = g->q_nst;
    h_info[12] = (int64_t)g->qcands.size();
    h_info[13] = g->cache.empty() ? 0 : (int64_t)g->cache.back().rounds.size();
    return FFB_OK;
}

extern "C" int ffb_group_quad_tuning(ffb_group_t g, int max, int *h_per_sm, int *h_stages, float *h_ms) {
    if (!g || max < 0) return FFB_ERR_ARG;
    const int n = std::min<int>(max, (int)g->qcands.size());
    for (int i = 0; i < n; ++i) {
        if (h_per_sm) h_per_sm[i] = g->qcands[i].per;
        if (h_stages) h_stages[i] = g->qcands[i].tile;
        if (h_ms) h_ms[i] = g->qcands[i].ms;
    }
    return n;
}

extern "C" int ffb_group_tuning(ffb_group_t g, int max, int *h_per, int *h_tile, int *h_grid, float *h_ms) {
    if (!g || max < 0) return FFB_ERR_ARG;
    const int m = std::min<int>(max, (int)g->cands.size());
    for (int i = 0; i < m; ++i) {
        if (h_per) h_per[i] = g->cands[i].per;
        if (h_tile) h_tile[i] = g->cands[i].tile;
        if (h_grid) h_grid[i] = g->cands[i].grid;
        if (h_ms) h_ms[i] = g->cands[i].ms;
    }
    return m;
}
