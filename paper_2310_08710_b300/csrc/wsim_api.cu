// Host side of the wsim C ABI (include/wsim.h).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "wsim_internal.h"

using namespace wsim;

struct RolloutKey {
    wsim_state st, traj;
    const float* act;
    const uint8_t* ctrl;
    wsim_metric_buf m;
    int t0, T, has_traj;
};

struct wsim_ctx {
    wsim_config cfg;
    wsim_batch b;
    Params p;
    int S = 0, N_tot = 0, grid = 1, count = 0;
    // scene-resident rollout: scenes in size buckets, each with a launch shape
    int shape_cap[kRollShapes] = {};   // staged segments per shape
    int cache_n = 32;                  // the largest scene's agents rounded up to a warp
    int shape_grid[kRollShapes] = {};  // persistent grid per shape
    int bucket_n[kBuckets] = {};       // scenes per bucket
    int bucket_at[kBuckets] = {};      // first entry of the bucket in border
    int bucket_shape[kBuckets] = {4, 0, 3};
    int split = 0, single_shape = 0;   // one launch of single_shape, or one per bucket
    int32_t* border = nullptr;         // cost-ordered scene ids, grouped by bucket
    cudaStream_t side[kBuckets] = {};
    cudaEvent_t fork = nullptr, join[kBuckets] = {};
    std::vector<int32_t> h_agent_off;
    // device scratch owned by the context
    int32_t *seg_off = nullptr, *seg_cnt = nullptr, *order = nullptr, *queue = nullptr, *status = nullptr;
    int queue_len = 0;
    float4* seg_geo = nullptr;
    float* seg_inv = nullptr;
    uint8_t* seg_flags = nullptr;
    float4* seg_tiles = nullptr;
    int32_t* seg_soff = nullptr;
    float4* seg_sup = nullptr;
    uint16_t* seg_tperm = nullptr;  // tiles in super-tile order, per scene
    int32_t* hint = nullptr;  // [N_tot][4] nearest-segment cache of the per-step kernels
    uint16_t* tlist = nullptr;  // [N_tot][kList] candidate-tile lists of the per-step kernels
    float4* tmeta = nullptr;    // [N_tot] their centre, radius and count
    float* route_rf = nullptr;  // [N_tot] each route's largest segment length over route_h
    unsigned long long* counters = nullptr;
    // observation: roadgraph point tiles, observer list, agent -> scene (built on first use)
    int32_t *pt_tile_off = nullptr, *pt_start = nullptr, *pt_cnt = nullptr, *obs_list = nullptr, *obs_count = nullptr,
            *scene_of = nullptr;
    float4* pt_box = nullptr;
    float* tmp = nullptr;  // ping-pong state, 10 x N_tot
    float* ckpt = nullptr;    // BPTT checkpoints
    float* segbuf = nullptr;  // BPTT recomputed segment states
    size_t ckpt_len = 0, seg_len = 0;
    // record of the differentiable rollout (wsim_rollout_record)
    float* rckpt = nullptr;     // its checkpoints
    int16_t* rec_ov = nullptr;  // [T][N_tot] deepest-overlap partners
    int32_t* rec_off = nullptr; // [T][N_tot] off-road records
    size_t rckpt_len = 0, rec_ov_len = 0, rec_off_len = 0;
    int rec_T = 0, rec_t0 = 0, rec_ck = 0, rec_metrics = 0;
    bool recorded = false;
    // captured rollout
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    RolloutKey key{};
    bool have_key = false;
    cudaStream_t last = nullptr;
};

namespace {

inline cudaStream_t S_(void* s) { return static_cast<cudaStream_t>(s); }

#define CK(expr)                                   \
    do {                                           \
        if ((expr) != cudaSuccess) {               \
            cudaGetLastError();                    \
            return WSIM_ECUDA;                     \
        }                                          \
    } while (0)

template <class T> int dalloc(T** p, size_t n) {
    if (n == 0) n = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return WSIM_ENOMEM;
    }
    return WSIM_OK;
}

bool state_ok(const wsim_state* s) {
    return s && s->x && s->y && s->x_lo && s->y_lo && s->th && s->th_lo && s->vx && s->vy && s->s && s->s_lo;
}
bool metrics_ok(const wsim_metric_buf* m) { return m && m->ov && m->off && m->logdiv && m->flags && m->reward; }

CStateP cstate(const wsim_state* s) {
    return CStateP{s->x, s->y, s->x_lo, s->y_lo, s->th, s->th_lo, s->vx, s->vy, s->s, s->s_lo};
}
StateP mstate(const wsim_state* s) {
    return StateP{s->x, s->y, s->x_lo, s->y_lo, s->th, s->th_lo, s->vx, s->vy, s->s, s->s_lo};
}
wsim_state offset(const wsim_state& s, size_t k) {
    return wsim_state{s.x + k, s.y + k, s.x_lo + k, s.y_lo + k, s.th + k,
                      s.th_lo + k, s.vx + k, s.vy + k, s.s + k, s.s_lo + k};
}
wsim_state tmp_state(const wsim_ctx* c) {
    float* t = c->tmp;
    size_t n = static_cast<size_t>(c->N_tot);
    return wsim_state{t, t + n, t + 2 * n, t + 3 * n, t + 4 * n, t + 5 * n, t + 6 * n, t + 7 * n, t + 8 * n, t + 9 * n};
}

StepArgs base_args(const wsim_ctx* c) {
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    const wsim_batch& b = c->b;
    a.S = b.S;
    a.N_tot = b.N_tot;
    a.T_log = b.T_log;
    a.agent_off = b.agent_off;
    a.L = b.L;
    a.W = b.W;
    a.v0 = b.idm_v0;
    a.valid = b.valid;
    a.kind = b.kind;
    a.route_off = b.route_off;
    a.route_x = b.route_x;
    a.route_y = b.route_y;
    a.route_rf = c->route_rf;
    a.log_x = b.log_x;
    a.log_y = b.log_y;
    a.log_th = b.log_th;
    a.log_vx = b.log_vx;
    a.log_vy = b.log_vy;
    a.segs = Segs{c->seg_off, c->seg_cnt, c->seg_geo, c->seg_inv, c->seg_flags, c->seg_tiles, c->seg_soff, c->seg_sup,
              c->seg_tperm};
    a.n_work = b.S;
    a.hint = c->hint;
    a.tlist = c->tlist;
    a.tmeta = c->tmeta;
    a.order = c->order;
    a.status = c->status;
    a.counters = c->counters;
    a.count = c->count;
    a.cache_n = c->cache_n;
    a.p = c->p;
    return a;
}

int ensure_queue(wsim_ctx* c, int n) {
    if (n <= c->queue_len) return WSIM_OK;
    if (c->exec) {  // the captured graph holds the old counters
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
        c->have_key = false;
    }
    if (c->queue) cudaFree(c->queue);
    c->queue = nullptr;
    c->queue_len = 0;
    int rc = dalloc(&c->queue, static_cast<size_t>(n));
    if (rc) return rc;
    c->queue_len = n;
    return WSIM_OK;
}

// One step (or metrics pass when in == out == nullptr for the transition).
int enqueue_step(wsim_ctx* c, const CStateP& in, const StateP* out, const float* act, const uint8_t* ctrl,
                 const wsim_metric_buf* m, int t_log, int32_t* queue, bool plain, cudaStream_t st) {
    StepArgs a = base_args(c);
    a.in = in;
    if (out) a.out = *out;
    a.act = act;
    a.ctrl = ctrl;
    a.do_transition = out != nullptr;
    a.do_metrics = m != nullptr;
    if (m) a.m = MetricsP{m->ov, m->off, m->logdiv, m->flags, m->reward};
    a.t_log = t_log;
    a.queue = queue;
    if (plain) {
        for (int s = 0; s < c->S; ++s) CK(launch_plain_scene(a, s, st));
    } else {
        CK(cudaMemsetAsync(queue, 0, sizeof(int32_t), st));
        CK(launch_step(a, c->grid, st));
    }
    return WSIM_OK;
}

int enqueue_rollout(wsim_ctx* c, const RolloutKey& k, bool plain, cudaStream_t st) {
    const size_t N = static_cast<size_t>(c->N_tot);
    const wsim_state tmp = tmp_state(c);
    wsim_state prev = k.st;
    for (int i = 0; i < k.T; ++i) {
        wsim_state out;
        if (k.has_traj)
            out = offset(k.traj, static_cast<size_t>(i) * N);
        else
            out = (i % 2 == 0) ? tmp : k.st;
        wsim_metric_buf m = k.m;
        m.ov += static_cast<size_t>(i) * N;
        m.off += static_cast<size_t>(i) * N;
        m.logdiv += static_cast<size_t>(i) * N;
        m.flags += static_cast<size_t>(i) * N;
        m.reward += static_cast<size_t>(i) * c->S;
        StateP o = mstate(&out);
        const float* act = k.act ? k.act + static_cast<size_t>(i) * 3 * N : nullptr;
        int rc = enqueue_step(c, cstate(&prev), &o, act, k.ctrl, &m, k.t0 + i + 1, c->queue + i, plain, st);
        if (rc) return rc;
        prev = out;
    }
    if (prev.x != k.st.x) {
        float* const src[10] = {prev.x, prev.y, prev.x_lo, prev.y_lo, prev.th, prev.th_lo, prev.vx, prev.vy, prev.s, prev.s_lo};
        float* const dst[10] = {k.st.x, k.st.y, k.st.x_lo, k.st.y_lo, k.st.th, k.st.th_lo, k.st.vx, k.st.vy, k.st.s, k.st.s_lo};
        for (int j = 0; j < 10; ++j) CK(cudaMemcpyAsync(dst[j], src[j], N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return WSIM_OK;
}

// Scene-resident rollout.  how: -1 = the context's configuration; a shape =
// whole batch with that shape; kHowSplit = one launch per bucket with the
// context's bucket shapes, concurrently; kHowBucket + kRollShapes*b + shape
// = bucket b alone with that shape.
constexpr int kHowSplit = 100, kHowBucket = 1000;

int enqueue_fused(wsim_ctx* c, const wsim_state* st, const float* act_seq, const uint8_t* ctrl, int t0, int T,
                  const wsim_metric_buf* mseq, const wsim_state* traj, int how, cudaStream_t s) {
    StepArgs a = base_args(c);
    a.in = cstate(st);
    a.out = mstate(st);
    a.act = act_seq;
    a.ctrl = ctrl;
    a.m = MetricsP{mseq->ov, mseq->off, mseq->logdiv, mseq->flags, mseq->reward};
    a.t_log = t0 + 1;
    a.T = T;
    if (traj) a.traj = mstate(traj);
    a.do_transition = 1;
    a.do_metrics = 1;
    if (how < 0) how = c->split ? kHowSplit : c->single_shape;
    CK(cudaMemsetAsync(c->queue, 0, kBuckets * sizeof(int32_t), s));
    if (how < kRollShapes) {  // whole batch, one shape
        a.order = c->order;
        a.n_work = c->S;
        a.queue = c->queue;
        a.seg_cap = c->shape_cap[how];
        CK(launch_rollout(how, a, std::min(c->S, c->shape_grid[how]), s));
        return WSIM_OK;
    }
    const bool split = how == kHowSplit;
    if (split) CK(cudaEventRecord(c->fork, s));
    for (int bk = 0; bk < kBuckets; ++bk) {
        if (c->bucket_n[bk] == 0) continue;
        int sh = c->bucket_shape[bk];
        if (!split) {
            if ((how - kHowBucket) / kRollShapes != bk) continue;
            sh = (how - kHowBucket) % kRollShapes;
        }
        a.order = c->border + c->bucket_at[bk];
        a.n_work = c->bucket_n[bk];
        a.queue = c->queue + bk;
        a.seg_cap = c->shape_cap[sh];
        cudaStream_t q = split ? c->side[bk] : s;
        if (split) CK(cudaStreamWaitEvent(q, c->fork, 0));
        CK(launch_rollout(sh, a, std::min(c->bucket_n[bk], c->shape_grid[sh]), q));
        if (split) {
            CK(cudaEventRecord(c->join[bk], q));
            CK(cudaStreamWaitEvent(s, c->join[bk], 0));
        }
    }
    return WSIM_OK;
}

}  // namespace

extern "C" {

void wsim_default_config(wsim_config* cfg) {
    if (!cfg) return;
    cfg->dt = 0.1f;
    cfg->idm_amax = 2.0f;
    cfg->idm_b = 3.0f;
    cfg->idm_T = 1.5f;
    cfg->idm_s0 = 2.0f;
    cfg->idm_dq = 2.0f;
    cfg->route_h = 0.5f;
    cfg->gap_min = 0.1f;
    cfg->loss_lambda = 1.0f;
    cfg->loss_tau = 0.25f;
    cfg->ckpt_every = 10;
    cfg->tile_segs = 0;
    cfg->kin_amax = 6.0f;
    cfg->kin_kmax = 0.3f;
    cfg->route_max_dist = 5.0f;
    cfg->route_max_rel = 2.0f;
    cfg->disc_a_max = 6.0f;
    cfg->disc_k_max = 0.3f;
    cfg->disc_d_max = 6.0f;
    cfg->disc_t_max = 0.3f;
    cfg->disc_na = 13;
    cfg->disc_nk = 31;
    cfg->disc_nd = 25;
    cfg->disc_nt = 13;
}

const char* wsim_strerror(int code) {
    switch (code) {
        case WSIM_OK: return "ok";
        case WSIM_EINVAL: return "invalid argument (null pointer, bad enum or inconsistent CSR offsets)";
        case WSIM_ESIZE: return "size outside the documented limits";
        case WSIM_ECUDA: return "a CUDA runtime call failed";
        case WSIM_ENONFINITE: return "a non-finite action or state reached a kernel";
        case WSIM_ETIMEOUT: return "a bounded device-side wait expired";
        case WSIM_ENOMEM: return "device allocation failed";
        case WSIM_ESTATE: return "call out of order";
        default: return "unknown wsim error";
    }
}

int wsim_init(wsim_ctx** out, const wsim_config* cfg, const wsim_batch* b, void* stream) {
    if (!out || !cfg || !b) return WSIM_EINVAL;
    *out = nullptr;
    if (b->S < 1 || b->N_tot < 0 || b->T_log < 2 || b->R_tot < 0 || b->route_tot < 0) return WSIM_ESIZE;
    if (!b->agent_off || !b->rg_off || !b->L || !b->W || !b->idm_v0 || !b->valid || !b->kind || !b->route_off ||
        !b->log_x || !b->log_y)
        return WSIM_EINVAL;
    if (b->R_tot > 0 && (!b->rg_x || !b->rg_y || !b->rg_poly || !b->rg_type || !b->rg_valid)) return WSIM_EINVAL;
    if (b->route_tot > 0 && (!b->route_x || !b->route_y)) return WSIM_EINVAL;
    if (!(cfg->dt > 0.f) || !(cfg->route_h > 0.f) || !(cfg->idm_amax > 0.f) || !(cfg->idm_b > 0.f))
        return WSIM_EINVAL;
    if (cfg->disc_na < 2 || cfg->disc_nk < 2 || cfg->disc_nd < 2 || cfg->disc_nt < 2 ||
        static_cast<int64_t>(cfg->disc_nd) * cfg->disc_nd * cfg->disc_nt > (1ll << 30) ||
        static_cast<int64_t>(cfg->disc_na) * cfg->disc_nk > (1ll << 30) || !(cfg->disc_a_max > 0.f) ||
        !(cfg->disc_k_max > 0.f) || !(cfg->disc_d_max > 0.f) || !(cfg->disc_t_max > 0.f))
        return WSIM_EINVAL;
    cudaStream_t st = S_(stream);
    const int S = b->S, N = b->N_tot;

    // Validate the CSR offsets and the IDM routes on the host.
    std::vector<int32_t> ao(S + 1), ro(S + 1), rto(static_cast<size_t>(N) + 1);
    std::vector<uint8_t> kind(static_cast<size_t>(N) + 1), valid(static_cast<size_t>(N) + 1);
    CK(cudaMemcpyAsync(ao.data(), b->agent_off, sizeof(int32_t) * (S + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ro.data(), b->rg_off, sizeof(int32_t) * (S + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rto.data(), b->route_off, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToHost, st));
    if (N > 0) {
        CK(cudaMemcpyAsync(kind.data(), b->kind, N, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(valid.data(), b->valid, N, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    if (ao[0] != 0 || ao[S] != N || ro[0] != 0 || ro[S] != b->R_tot || rto[0] != 0 || rto[N] != b->route_tot)
        return WSIM_EINVAL;
    for (int s = 0; s < S; ++s) {
        const int n = ao[s + 1] - ao[s];
        if (n < 0 || ro[s + 1] < ro[s]) return WSIM_EINVAL;
        if (n > WSIM_MAX_AGENTS) return WSIM_ESIZE;
    }
    for (int g = 0; g < N; ++g) {
        if (rto[g + 1] < rto[g]) return WSIM_EINVAL;
        if (kind[g] > WSIM_KIND_IDM) return WSIM_EINVAL;
        if (kind[g] == WSIM_KIND_IDM && valid[g] && rto[g + 1] - rto[g] < 2) return WSIM_EINVAL;
    }

    wsim_ctx* c = new wsim_ctx();
    c->cfg = *cfg;
    c->b = *b;
    c->S = S;
    c->N_tot = N;
    c->h_agent_off = ao;
    c->p = Params{cfg->dt,     cfg->idm_amax,         cfg->idm_b,  cfg->idm_T,
                  cfg->idm_s0, cfg->idm_dq,           cfg->route_h, 1.0f / cfg->route_h,
                  cfg->gap_min, 2.0f * sqrtf(cfg->idm_amax * cfg->idm_b), 1.0f / cfg->dt, cfg->kin_amax, cfg->kin_kmax,
                  cfg->disc_a_max, cfg->disc_k_max, cfg->disc_d_max, cfg->disc_t_max,
                  cfg->disc_na, cfg->disc_nk, cfg->disc_nd, cfg->disc_nt};
    int rc = WSIM_OK;
    auto fail = [&](int code) {
        wsim_destroy(c);
        return code;
    };
    if ((rc = dalloc(&c->seg_off, S + 1)) || (rc = dalloc(&c->seg_cnt, S)) || (rc = dalloc(&c->order, S)) ||
        (rc = dalloc(&c->border, S)) ||
        (rc = dalloc(&c->status, 1)) || (rc = dalloc(&c->counters, kCounters)) ||
        (rc = dalloc(&c->tmp, static_cast<size_t>(N) * 10)) || (rc = ensure_queue(c, 128)) ||
        (rc = dalloc(&c->hint, static_cast<size_t>(N) * 4)) ||
        (rc = dalloc(&c->tlist, static_cast<size_t>(N) * kList)) || (rc = dalloc(&c->tmeta, static_cast<size_t>(N))) ||
        (rc = dalloc(&c->route_rf, static_cast<size_t>(N))))
        return fail(rc);
    if (launch_route_speed(b->route_off, b->route_x, b->route_y, N, 1.0f / cfg->route_h, c->route_rf, st) !=
        cudaSuccess)
        return fail(WSIM_ECUDA);
    // all-ones: no nearest segment known, list count -1 (no list yet)
    if (cudaMemsetAsync(c->hint, 0xff, std::max<size_t>(N, 1) * 4 * sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(c->tmeta, 0xff, std::max<size_t>(N, 1) * sizeof(float4), st) != cudaSuccess)
        return fail(WSIM_ECUDA);
    if (cudaMemsetAsync(c->status, 0, sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(c->counters, 0, kCounters * sizeof(unsigned long long), st) != cudaSuccess)
        return fail(WSIM_ECUDA);

    // Road-edge segments: count, pad each scene to kSegAlign, pack.
    if (launch_seg_count(b->rg_off, b->rg_x, b->rg_y, b->rg_poly, b->rg_type, b->rg_valid, S, c->seg_cnt, st) !=
        cudaSuccess)
        return fail(WSIM_ECUDA);
    std::vector<int32_t> cnt(S), off(S + 1, 0);
    if (cudaMemcpyAsync(cnt.data(), c->seg_cnt, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(WSIM_ECUDA);
    std::vector<int32_t> soff(S + 1, 0);
    int64_t padded = 0;  // packed positions are int32 indexes; tile lists hold 16-bit tile indexes
    for (int s = 0; s < S; ++s) {
        padded += ((static_cast<int64_t>(cnt[s]) + kSegAlign - 1) / kSegAlign) * kSegAlign;
        if (cnt[s] > kMaxSceneSegs) return fail(WSIM_ESIZE);
    }
    if (padded > INT32_MAX) return fail(WSIM_ESIZE);
    for (int s = 0; s < S; ++s) {
        off[s + 1] = off[s] + ((cnt[s] + kSegAlign - 1) / kSegAlign) * kSegAlign;
        const int nt = (cnt[s] + kTile - 1) / kTile;
        soff[s + 1] = soff[s] + (nt + kSuper - 1) / kSuper;
    }
    const size_t E = static_cast<size_t>(off[S]);
    if ((rc = dalloc(&c->seg_geo, E)) || (rc = dalloc(&c->seg_inv, E)) || (rc = dalloc(&c->seg_flags, E)) ||
        (rc = dalloc(&c->seg_tiles, 2 * (E / kTile))) || (rc = dalloc(&c->seg_soff, S + 1)) ||
        (rc = dalloc(&c->seg_sup, static_cast<size_t>(soff[S]))) ||
        (rc = dalloc(&c->seg_tperm, std::max<size_t>(E / kTile, 1))))
        return fail(rc);
    if (cudaMemcpyAsync(c->seg_soff, soff.data(), sizeof(int32_t) * (S + 1), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return fail(WSIM_ECUDA);
    if (cudaMemsetAsync(c->seg_geo, 0, std::max<size_t>(E, 1) * sizeof(float4), st) != cudaSuccess ||
        cudaMemsetAsync(c->seg_inv, 0, std::max<size_t>(E, 1) * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(c->seg_flags, 0, std::max<size_t>(E, 1), st) != cudaSuccess ||
        cudaMemcpyAsync(c->seg_off, off.data(), sizeof(int32_t) * (S + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(WSIM_ECUDA);
    if (launch_seg_pack(b->rg_off, b->rg_x, b->rg_y, b->rg_poly, b->rg_type, b->rg_valid, S, c->seg_off, c->seg_geo,
                        c->seg_inv, c->seg_flags, st) != cudaSuccess ||
        launch_tile_build(S, c->seg_off, c->seg_cnt, c->seg_geo, c->seg_flags, c->seg_tiles, st) != cudaSuccess ||
        launch_tile_order(S, c->seg_off, c->seg_cnt, c->seg_tiles, c->seg_tperm, st) != cudaSuccess ||
        launch_super_build(S, c->seg_off, c->seg_cnt, c->seg_soff, c->seg_tiles, c->seg_tperm, c->seg_sup, st) !=
            cudaSuccess)
        return fail(WSIM_ECUDA);

    // Scene work list, most expensive first (longest-processing-time order).
    std::vector<double> cost(S);
    for (int s = 0; s < S; ++s) {
        const double n = ao[s + 1] - ao[s];
        cost[s] = 4.0 * n * cnt[s] + 32.0 * n * n + 64.0;
    }
    std::vector<int32_t> order(S);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    if (cudaMemcpyAsync(c->order, order.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(WSIM_ECUDA);

    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->grid = std::min(S, sms * step_blocks_per_sm());
    // Scene-resident rollout.  Buckets by staged size: 0 = fits the small
    // stage (shapes 1 and 4), 1 = fits the large stage (shape 0), 2 = neither.
    int need = 0, nmax = 1;
    for (int s = 0; s < S; ++s) {
        need = std::max(need, off[s + 1] - off[s]);
        nmax = std::max(nmax, ao[s + 1] - ao[s]);
    }
    c->cache_n = std::min(kMaxN, (nmax + 31) / 32 * 32);
    for (int sh = 0; sh < kRollShapes; ++sh) c->shape_cap[sh] = std::min(need, shape_max_seg_cap(sh, c->cache_n));
    std::vector<int32_t> border;
    for (int bk = 0; bk < kBuckets; ++bk) {
        c->bucket_at[bk] = static_cast<int>(border.size());
        for (int w = 0; w < S; ++w) {
            const int s = order[w], segs = off[s + 1] - off[s];
            const int b = segs <= shape_max_seg_cap(1, c->cache_n) ? 0 : (segs <= shape_max_seg_cap(0, c->cache_n) ? 1 : 2);
            if (b == bk) border.push_back(s);
        }
        c->bucket_n[bk] = static_cast<int>(border.size()) - c->bucket_at[bk];
    }
    for (int sh = 0; sh < kRollShapes; ++sh) {
        int bps = 1;
        if (shape_prepare(sh, c->shape_cap[sh], c->cache_n, &bps) != cudaSuccess) return fail(WSIM_ECUDA);
        c->shape_grid[sh] = sms * bps;
    }
    if (cudaMemcpyAsync(c->border, border.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(WSIM_ECUDA);
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(WSIM_ECUDA);
    for (int b = 0; b < kBuckets; ++b)
        if (cudaStreamCreateWithFlags(&c->side[b], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->join[b], cudaEventDisableTiming) != cudaSuccess)
            return fail(WSIM_ECUDA);
    // Default until tuned: one launch of 512 x 2 CTAs per SM, with the scenes'
    // segments staged in shared memory if every scene fits the stage.
    c->single_shape = c->bucket_n[1] + c->bucket_n[2] > 0 ? 3 : 4;
    c->last = st;
    *out = c;
    return WSIM_OK;
}

int wsim_step(wsim_ctx* c, const wsim_state* in, const float* act, const uint8_t* ctrl, wsim_state* out,
              const wsim_metric_buf* m, int t, void* stream) {
    if (!c || !state_ok(in) || !state_ok(out) || (!act && !ctrl) || (m && !metrics_ok(m))) return WSIM_EINVAL;
    if (in->x == out->x) return WSIM_EINVAL;
    if (t < 0 || t + 1 >= c->b.T_log) return WSIM_ESIZE;
    c->last = S_(stream);
    StateP o = mstate(out);
    return enqueue_step(c, cstate(in), &o, act, ctrl, m, t + 1, c->queue, false, S_(stream));
}

int wsim_metrics(wsim_ctx* c, const wsim_state* st, const wsim_metric_buf* m, int t, void* stream) {
    if (!c || !state_ok(st) || !metrics_ok(m)) return WSIM_EINVAL;
    if (t < 0 || t >= c->b.T_log) return WSIM_ESIZE;
    c->last = S_(stream);
    return enqueue_step(c, cstate(st), nullptr, nullptr, nullptr, m, t, c->queue, false, S_(stream));
}

int wsim_rollout(wsim_ctx* c, wsim_state* st, const float* act_seq, const uint8_t* ctrl, int t0, int T, int mode,
                 const wsim_metric_buf* mseq, const wsim_state* traj, void* stream) {
    if (!c || !state_ok(st) || (!act_seq && !ctrl) || !metrics_ok(mseq) || (traj && !state_ok(traj)))
        return WSIM_EINVAL;
    if (mode < WSIM_MODE_GRAPH || mode > WSIM_MODE_FUSED) return WSIM_EINVAL;
    if (T < 1 || t0 < 0 || t0 + T >= c->b.T_log) return WSIM_ESIZE;
    cudaStream_t s = S_(stream);
    c->last = s;
    int rc = ensure_queue(c, T);
    if (rc) return rc;
    RolloutKey k{};
    std::memset(&k, 0, sizeof(k));
    k.st = *st;
    if (traj) k.traj = *traj;
    k.act = act_seq;
    k.ctrl = ctrl;
    k.m = *mseq;
    k.t0 = t0;
    k.T = T;
    k.has_traj = traj != nullptr;
    if (mode == WSIM_MODE_FUSED) return enqueue_fused(c, st, act_seq, ctrl, t0, T, mseq, traj, -1, s);
    if (mode != WSIM_MODE_GRAPH) return enqueue_rollout(c, k, mode == WSIM_MODE_PLAIN, s);

    if (!c->exec || !c->have_key || std::memcmp(&k, &c->key, sizeof(k)) != 0) {
        if (c->exec) {
            cudaGraphExecDestroy(c->exec);
            c->exec = nullptr;
        }
        c->have_key = false;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_rollout(c, k, false, c->cap);
        cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc ? rc : WSIM_ECUDA;
        }
        e = cudaGraphInstantiate(&c->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->exec = nullptr;
            return WSIM_ECUDA;
        }
        c->key = k;
        c->have_key = true;
    }
    CK(cudaGraphLaunch(c->exec, s));
    return WSIM_OK;
}

int wsim_discretize(wsim_ctx* c, const float* act, int T, int32_t* idx, void* stream) {
    if (!c || !act || !idx) return WSIM_EINVAL;
    if (T < 0) return WSIM_ESIZE;
    c->last = S_(stream);
    CK(launch_discretize(base_args(c), act, T, idx, S_(stream)));
    return WSIM_OK;
}

int wsim_decode_actions(wsim_ctx* c, const int32_t* idx, int T, float* act, void* stream) {
    if (!c || !act || !idx) return WSIM_EINVAL;
    if (T < 0) return WSIM_ESIZE;
    c->last = S_(stream);
    CK(launch_decode_actions(base_args(c), idx, T, act, S_(stream)));
    return WSIM_OK;
}

int wsim_route_metrics(wsim_ctx* c, const wsim_state* st, float* progress, uint8_t* off_route, void* stream) {
    if (!c || !state_ok(st) || !progress || !off_route) return WSIM_EINVAL;
    const wsim_batch& b = c->b;
    if (!b.path_off || !b.path_pt_off || !b.path_x || !b.path_y || !b.path_on) return WSIM_EINVAL;
    c->last = S_(stream);
    StepArgs a = base_args(c);
    a.in = cstate(st);
    CK(launch_route(a, b.path_off, b.path_pt_off, b.path_x, b.path_y, b.path_on, c->cfg.route_max_dist,
                    c->cfg.route_max_rel, progress, off_route, S_(stream)));
    return WSIM_OK;
}

int wsim_observe(wsim_ctx* c, const wsim_state* st, const uint8_t* observers, int M, int K, float* agents,
                 uint8_t* agents_valid, float* rg, int32_t* rg_idx, void* stream) {
    if (!c || !state_ok(st) || !agents || !agents_valid || !rg || !rg_idx) return WSIM_EINVAL;
    int nmax = 0;
    for (int s = 0; s < c->S; ++s) nmax = std::max(nmax, c->h_agent_off[s + 1] - c->h_agent_off[s]);
    if (M < nmax || M < 1 || K < 1 || K > WSIM_OBS_MAX_K) return WSIM_ESIZE;
    cudaStream_t s = S_(stream);
    c->last = s;
    if (!c->pt_box) {  // first call: point tiles and the agent -> scene map
        const int S = c->S, N = c->N_tot;
        std::vector<int32_t> cnt(S), toff(S + 1, 0), sc(std::max(N, 1));
        int32_t* dcnt = nullptr;
        int rc = dalloc(&dcnt, S);
        if (rc) return rc;
        // tiles per scene (runs of one polyline, at most kPtTile points each)
        cudaError_t e = launch_pt_count(c->b.rg_off, c->b.rg_poly, S, dcnt, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(dcnt);
        CK(e);
        for (int i = 0; i < S; ++i) toff[i + 1] = toff[i] + cnt[i];
        for (int i = 0; i < S; ++i)
            for (int g = c->h_agent_off[i]; g < c->h_agent_off[i + 1]; ++g) sc[g] = i;
        if ((rc = dalloc(&c->pt_tile_off, S + 1)) || (rc = dalloc(&c->pt_start, toff[S] + 1)) ||
            (rc = dalloc(&c->pt_cnt, toff[S])) || (rc = dalloc(&c->pt_box, toff[S])) ||
            (rc = dalloc(&c->obs_list, 2 * N)) || (rc = dalloc(&c->obs_count, 3)) || (rc = dalloc(&c->scene_of, N))) {
            cudaFree(c->pt_tile_off);
            cudaFree(c->pt_start);
            cudaFree(c->pt_cnt);
            cudaFree(c->pt_box);
            cudaFree(c->obs_list);
            cudaFree(c->obs_count);
            cudaFree(c->scene_of);
            c->pt_tile_off = c->pt_start = c->pt_cnt = c->obs_list = c->obs_count = c->scene_of = nullptr;
            c->pt_box = nullptr;
            return rc;
        }
        CK(cudaMemcpyAsync(c->pt_tile_off, toff.data(), sizeof(int32_t) * (S + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->scene_of, sc.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
        CK(launch_pt_tiles(c->b.rg_off, c->b.rg_poly, c->pt_tile_off, c->b.rg_x, c->b.rg_y, c->b.rg_valid, S,
                           c->pt_start, c->pt_box, c->pt_cnt, s));
        CK(cudaStreamSynchronize(s));
    }
    StepArgs a = base_args(c);
    a.in = cstate(st);
    CK(launch_observe(a, observers, c->obs_list, c->obs_count, c->b.rg_x, c->b.rg_y, c->b.rg_valid, c->pt_tile_off,
                      c->pt_start, c->pt_box, c->pt_cnt, c->scene_of, M, K, agents, agents_valid, rg, rg_idx, s));
    return WSIM_OK;
}

int wsim_expert_actions(wsim_ctx* c, int t0, int T, float* act_out, void* stream) {
    if (!c || !act_out) return WSIM_EINVAL;
    if (!c->b.log_th || !c->b.log_vx || !c->b.log_vy) return WSIM_EINVAL;
    if (t0 < 0 || T < 0 || t0 + T >= c->b.T_log) return WSIM_ESIZE;
    c->last = S_(stream);
    CK(launch_expert_actions(base_args(c), t0, T, act_out, S_(stream)));
    return WSIM_OK;
}

int wsim_autotune(wsim_ctx* c, const wsim_state* st, const float* act_seq, int t0, int T, wsim_tuning* out,
                  void* stream) {
    if (!c || !state_ok(st) || !act_seq || !out) return WSIM_EINVAL;
    if (T < 1 || t0 < 0 || t0 + T >= c->b.T_log) return WSIM_ESIZE;
    cudaStream_t s = S_(stream);
    c->last = s;
    int rc = ensure_queue(c, 128);
    if (rc) return rc;
    const size_t N = static_cast<size_t>(c->N_tot), S = static_cast<size_t>(c->S);
    // Scratch metric rows for T steps; the caller's state is copied, not changed.
    unsigned char* buf = nullptr;
    const size_t bytes = static_cast<size_t>(T) * (N * (3 * sizeof(float) + 1) + S * sizeof(int32_t)) + 64;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WSIM_ENOMEM;
    }
    wsim_metric_buf m;
    float* f = reinterpret_cast<float*>(buf);
    m.ov = f;
    m.off = f + T * N;
    m.logdiv = f + 2 * T * N;
    m.reward = reinterpret_cast<int32_t*>(f + 3 * T * N);
    m.flags = reinterpret_cast<uint8_t*>(m.reward + T * S);
    const wsim_state tmp = tmp_state(c);
    float* const src[10] = {st->x, st->y, st->x_lo, st->y_lo, st->th, st->th_lo, st->vx, st->vy, st->s, st->s_lo};
    float* const dst[10] = {tmp.x, tmp.y, tmp.x_lo, tmp.y_lo, tmp.th, tmp.th_lo, tmp.vx, tmp.vy, tmp.s, tmp.s_lo};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WSIM_ECUDA;
    // Time one configuration (first run warms up).
    auto timeit = [&](int how, float* ms) {
        for (int rep = 0; rep < 2 && rc == WSIM_OK; ++rep) {
            for (int j = 0; j < 10; ++j)
                if (cudaMemcpyAsync(dst[j], src[j], N * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    rc = WSIM_ECUDA;
            if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = WSIM_ECUDA;
            if (!rc) rc = enqueue_fused(c, &tmp, act_seq, nullptr, t0, T, &m, nullptr, how, s);
            if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
                rc = WSIM_ECUDA;
        }
    };
    std::memset(out, 0, sizeof(*out));
    float best = 1e30f;
    int best_how = 0;
    for (int sh = 0; sh < kRollShapes; ++sh) {
        out->ms_single[sh] = -1.f;
        timeit(sh, &out->ms_single[sh]);
        if (!rc && out->ms_single[sh] < best) {
            best = out->ms_single[sh];
            best_how = sh;
        }
    }
    int used = 0;
    for (int bk = 0; bk < kBuckets; ++bk) {
        out->bucket_scenes[bk] = c->bucket_n[bk];
        float bb = 1e30f;
        for (int sh = 0; sh < kRollShapes; ++sh) {
            out->ms_bucket[bk][sh] = -1.f;
            if (!c->bucket_n[bk] || rc) continue;
            timeit(kHowBucket + kRollShapes * bk + sh, &out->ms_bucket[bk][sh]);
            if (!rc && out->ms_bucket[bk][sh] < bb) {
                bb = out->ms_bucket[bk][sh];
                c->bucket_shape[bk] = sh;
            }
        }
        used += c->bucket_n[bk] > 0;
    }
    out->ms_split = -1.f;
    if (used > 1 && !rc) {
        timeit(kHowSplit, &out->ms_split);
        if (!rc && out->ms_split < best) {
            best = out->ms_split;
            best_how = kHowSplit;
        }
    }
    if (!rc) {
        c->split = best_how == kHowSplit;
        if (!c->split) c->single_shape = best_how;
    }
    out->split = c->split;
    out->single_shape = c->single_shape;
    for (int bk = 0; bk < kBuckets; ++bk) out->bucket_shape[bk] = c->bucket_shape[bk];
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (rc) cudaGetLastError();
    return rc;
}

int wsim_set_tuning(wsim_ctx* c, const wsim_tuning* t) {
    if (!c || !t) return WSIM_EINVAL;
    if (t->single_shape < 0 || t->single_shape >= kRollShapes) return WSIM_EINVAL;
    for (int b = 0; b < kBuckets; ++b)
        if (t->bucket_shape[b] < 0 || t->bucket_shape[b] >= kRollShapes) return WSIM_EINVAL;
    c->split = t->split ? 1 : 0;
    c->single_shape = t->single_shape;
    for (int b = 0; b < kBuckets; ++b) c->bucket_shape[b] = t->bucket_shape[b];
    return WSIM_OK;
}

int wsim_get_tuning(wsim_ctx* c, wsim_tuning* out) {
    if (!c || !out) return WSIM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->split = c->split;
    out->single_shape = c->single_shape;
    for (int k = 0; k < kRollShapes; ++k) out->ms_single[k] = -1.f;
    for (int b = 0; b < kBuckets; ++b) {
        out->bucket_shape[b] = c->bucket_shape[b];
        out->bucket_scenes[b] = c->bucket_n[b];
        for (int k = 0; k < kRollShapes; ++k) out->ms_bucket[b][k] = -1.f;
    }
    out->ms_split = -1.f;
    return WSIM_OK;
}

}  // extern "C"

namespace {

// Grows a scratch array of the context to at least `need` elements
// (synchronises the stream first: a kernel may still use the old one).
template <class T> int grow(T** p, size_t* len, size_t need, cudaStream_t s) {
    if (need <= *len) return WSIM_OK;
    CK(cudaStreamSynchronize(s));
    cudaFree(*p);
    *p = nullptr;
    *len = 0;
    int rc = dalloc(p, need);
    if (rc) return rc;
    *len = need;
    return WSIM_OK;
}

int bptt_grid(const wsim_ctx* c, int which) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::min(c->S, sms * bptt_blocks_per_sm(which));
}

}  // namespace

extern "C" {

int wsim_rollout_record(wsim_ctx* c, const wsim_state* st0, const float* act_seq, int t0, int T, int ckpt_every,
                        const wsim_metric_buf* mseq, double* loss, wsim_state* st_T, void* stream) {
    if (!c || !state_ok(st0) || !act_seq || (mseq && !metrics_ok(mseq)) || (st_T && !state_ok(st_T)))
        return WSIM_EINVAL;
    if (st_T && st_T->x == st0->x) return WSIM_EINVAL;
    if (T < 1 || t0 < 0 || t0 + T >= c->b.T_log || ckpt_every < 1) return WSIM_ESIZE;
    cudaStream_t s = S_(stream);
    c->last = s;
    c->recorded = false;
    const int ck = std::min(ckpt_every, T);
    const size_t per = 10 * static_cast<size_t>(c->N_tot);
    const size_t rows = static_cast<size_t>(T) * static_cast<size_t>(c->N_tot);
    int rc = grow(&c->rckpt, &c->rckpt_len, static_cast<size_t>((T + ck - 1) / ck + 1) * per, s);
    if (rc) return rc;
    if (mseq && ((rc = grow(&c->rec_ov, &c->rec_ov_len, rows, s)) || (rc = grow(&c->rec_off, &c->rec_off_len, rows, s))))
        return rc;
    StepArgs a = base_args(c);
    a.in = cstate(st0);
    if (st_T) a.out = mstate(st_T);
    a.act = act_seq;
    a.t_log = t0 + 1;
    a.T = T;
    a.queue = c->queue;
    a.do_transition = 1;
    a.do_metrics = mseq != nullptr;
    if (mseq) a.m = MetricsP{mseq->ov, mseq->off, mseq->logdiv, mseq->flags, mseq->reward};
    CK(cudaMemsetAsync(c->queue, 0, sizeof(int32_t), s));
    CK(launch_record(a, c->rckpt, ck, loss, mseq != nullptr, c->rec_ov, c->rec_off, c->cfg.loss_lambda,
                     c->cfg.loss_tau, bptt_grid(c, 1), s));
    c->rec_T = T;
    c->rec_t0 = t0;
    c->rec_ck = ck;
    c->rec_metrics = mseq != nullptr;
    c->recorded = true;
    return WSIM_OK;
}

int wsim_rollout_backward(wsim_ctx* c, const float* act_seq, const wsim_metric_grad* gm, const double* loss_w,
                          float* dact, wsim_state* dst0, void* stream) {
    if (!c || !act_seq || (!dact && !dst0) || (dst0 && !state_ok(dst0))) return WSIM_EINVAL;
    if (!c->recorded) return WSIM_ESTATE;
    const bool metrics = gm && (gm->logdiv || gm->ov || gm->off);
    if (metrics && !c->rec_metrics) return WSIM_ESTATE;
    cudaStream_t s = S_(stream);
    c->last = s;
    const int T = c->rec_T, ck = c->rec_ck;
    int rc = grow(&c->segbuf, &c->seg_len, static_cast<size_t>(ck + 1) * 10 * static_cast<size_t>(c->N_tot), s);
    if (rc) return rc;
    StepArgs a = base_args(c);
    a.act = act_seq;
    a.t_log = c->rec_t0 + 1;
    a.T = T;
    a.queue = c->queue;
    a.do_transition = 1;
    StateP d{};
    if (dst0) d = mstate(dst0);
    CK(cudaMemsetAsync(c->queue, 0, sizeof(int32_t), s));
    CK(launch_backward(a, c->rckpt, c->segbuf, ck, c->rec_ov, c->rec_off, metrics ? gm->logdiv : nullptr,
                       metrics ? gm->ov : nullptr, metrics ? gm->off : nullptr, loss_w, dact, d, c->cfg.loss_lambda,
                       c->cfg.loss_tau, bptt_grid(c, 0), s));
    return WSIM_OK;
}

int wsim_loss_grad(wsim_ctx* c, const wsim_state* st0, const float* act_seq, int t0, int T, int ckpt_every,
                   int flags, double* loss, float* dact, void* stream) {
    if (!c || !state_ok(st0) || !act_seq || !loss) return WSIM_EINVAL;
    if (T < 1 || t0 < 0 || t0 + T >= c->b.T_log || ckpt_every < 1) return WSIM_ESIZE;
    if (flags & ~WSIM_GRAD_PLAIN) return WSIM_EINVAL;
    cudaStream_t s = S_(stream);
    c->last = s;
    const int ck = std::min(ckpt_every, T);
    const size_t per = 10 * static_cast<size_t>(c->N_tot);
    const size_t nck = static_cast<size_t>((T + ck - 1) / ck + 1) * per, nsg = static_cast<size_t>(ck + 1) * per;
    if (nck > c->ckpt_len) {
        CK(cudaStreamSynchronize(s));
        cudaFree(c->ckpt);
        c->ckpt = nullptr;
        c->ckpt_len = 0;
        int rc = dalloc(&c->ckpt, nck);
        if (rc) return rc;
        c->ckpt_len = nck;
    }
    if (nsg > c->seg_len) {
        CK(cudaStreamSynchronize(s));
        cudaFree(c->segbuf);
        c->segbuf = nullptr;
        c->seg_len = 0;
        int rc = dalloc(&c->segbuf, nsg);
        if (rc) return rc;
        c->seg_len = nsg;
    }
    StepArgs a = base_args(c);
    a.in = cstate(st0);
    a.act = act_seq;
    a.t_log = t0 + 1;
    a.T = T;
    a.queue = c->queue;
    a.do_transition = 1;
    const bool plain = (flags & WSIM_GRAD_PLAIN) != 0;
    if (!plain) CK(cudaMemsetAsync(c->queue, 0, sizeof(int32_t), s));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    CK(launch_bptt(a, c->ckpt, c->segbuf, ck, loss, dact, c->cfg.loss_lambda, c->cfg.loss_tau,
                   std::min(c->S, sms * bptt_blocks_per_sm()), plain, s));
    return WSIM_OK;
}

int wsim_status(wsim_ctx* c, int* device_status, void* stream) {
    if (!c || !device_status) return WSIM_EINVAL;
    cudaStream_t s = S_(stream);
    int v = 0;
    CK(cudaMemcpyAsync(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    *device_status = v;
    return WSIM_OK;
}

int wsim_set_counting(wsim_ctx* c, int on) {
    if (!c) return WSIM_EINVAL;
    c->count = on ? 1 : 0;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
        c->have_key = false;
    }
    CK(cudaMemsetAsync(c->counters, 0, kCounters * sizeof(unsigned long long), c->last));
    return WSIM_OK;
}

int wsim_counters(wsim_ctx* c, int64_t out[WSIM_COUNTERS], void* stream) {
    if (!c || !out) return WSIM_EINVAL;
    unsigned long long v[kCounters];
    cudaStream_t s = S_(stream);
    CK(cudaMemcpyAsync(v, c->counters, sizeof(v), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < kCounters; ++k) out[k] = static_cast<int64_t>(v[k]);
    return WSIM_OK;
}

void wsim_destroy(wsim_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->last);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->fork) cudaEventDestroy(c->fork);
    for (int b = 0; b < kBuckets; ++b) {
        if (c->side[b]) cudaStreamDestroy(c->side[b]);
        if (c->join[b]) cudaEventDestroy(c->join[b]);
    }
    cudaFree(c->seg_off);
    cudaFree(c->seg_cnt);
    cudaFree(c->order);
    cudaFree(c->border);
    cudaFree(c->queue);
    cudaFree(c->status);
    cudaFree(c->counters);
    cudaFree(c->pt_tile_off);
    cudaFree(c->pt_start);
    cudaFree(c->pt_cnt);
    cudaFree(c->pt_box);
    cudaFree(c->obs_list);
    cudaFree(c->obs_count);
    cudaFree(c->scene_of);
    cudaFree(c->tmp);
    cudaFree(c->ckpt);
    cudaFree(c->segbuf);
    cudaFree(c->rckpt);
    cudaFree(c->rec_ov);
    cudaFree(c->rec_off);
    cudaFree(c->seg_geo);
    cudaFree(c->seg_inv);
    cudaFree(c->seg_flags);
    cudaFree(c->seg_tiles);
    cudaFree(c->seg_soff);
    cudaFree(c->seg_sup);
    cudaFree(c->seg_tperm);
    cudaFree(c->hint);
    cudaFree(c->tlist);
    cudaFree(c->tmeta);
    cudaFree(c->route_rf);
    delete c;
}

}  // extern "C"
