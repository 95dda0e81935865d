// wsim per-step kernels (sm_103a) and the road-edge packing kernels of
// wsim_init.
//
// Per step, one CTA owns one scene at a time.  The step kernel is
// persistent: its CTAs take scene ids from an atomic work counter over a
// cost-ordered list, so scenes of uneven size share one launch.  Per scene:
//   transition  (Sec. 4 step): IDM agents in groups of eight per warp (the
//               lead search warp-wide with one look-ahead sample per lane,
//               acceleration and route advance one lane per agent, Sec. 3.5),
//               policy agents one per thread (bicycle / delta dynamics,
//               App. A.1), compensated positions;
//   overlap     (Sec. 3.4 collision): pairs from shared-memory boxes, culled
//               exactly, one warp per row;
//   off-road    (Sec. 3.4 off-road): culled nearest-segment search per box
//               corner, eight agents per warp (one lane per corner) with
//               per-agent candidate-tile lists and last winners, segments
//               read from global memory, a warp-cooperative full search
//               when the cache cannot prove the answer;
//   finish      log divergence (Sec. 3.4), flags and the sparse reward
//               (Sec. 5.2).
// The plain path runs the same phases as separate one-CTA launches per scene.
#include "wsim_phases.cuh"

namespace wsim {

constexpr int NTs = kStepThreads;

// COUNT = false: the work counts are dead code (fewer live registers).
// Both instantiations are held to 64 registers (4 CTAs of 256 per SM): the
// graph path sizes its grid by the smaller occupancy of the two.
template <bool COUNT>
__global__ void __launch_bounds__(NTs, 4) k_step(const StepArgs A) {
    __shared__ AgentSmem sm;
    init_cta(sm);
    Counts cnt;
    for (;;) {
        if (threadIdx.x == 0) sm.scene = atomicAdd(A.queue, 1);
        __syncthreads();
        const int w = sm.scene;
        if (w >= A.n_work) break;
        const int s = A.order[w];
        const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
        load_state<NTs>(sm, A, A.in, a0, N);
        __syncthreads();
        if (A.do_transition) {
            phase_transition<NTs>(sm, A, A.act, A.t_log, a0, N, cnt);
            __syncthreads();
            writeback<NTs>(sm, A.p, &A.out, a0, N);
            __syncthreads();
        }
        if (A.do_metrics) {
            const SegView V = global_view(A.segs, s);
            phase_metrics<NTs>(sm, V, A.hint ? A.hint + 4 * a0 : nullptr, A.tlist ? A.tlist + kList * a0 : nullptr,
                               A.tmeta ? A.tmeta + a0 : nullptr, N, true, true, kListLook * A.p.dt, cnt);
            __syncthreads();
            phase_finish<NTs>(sm, A, A.m, A.m.reward + s, A.t_log, a0, N);
        }
        __syncthreads();
    }
    if (COUNT) publish_counts(sm, A, cnt);
}

// ---------------------------------------------------------------------------
// Plain path: one single-CTA launch per scene and phase.
// ---------------------------------------------------------------------------
__device__ __forceinline__ CStateP as_const(const StateP& s) {
    return CStateP{s.x, s.y, s.x_lo, s.y_lo, s.th, s.th_lo, s.vx, s.vy, s.s, s.s_lo};
}

__global__ void __launch_bounds__(NTs) k_plain_transition(const StepArgs A, int s) {
    __shared__ AgentSmem sm;
    init_cta(sm);
    Counts cnt;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    load_state<NTs>(sm, A, A.in, a0, N);
    __syncthreads();
    phase_transition<NTs>(sm, A, A.act, A.t_log, a0, N, cnt);
    __syncthreads();
    writeback<NTs>(sm, A.p, &A.out, a0, N);
    publish_counts(sm, A, cnt);
}

__global__ void __launch_bounds__(NTs) k_plain_overlap(const StepArgs A, int s) {
    __shared__ AgentSmem sm;
    init_cta(sm);
    Counts cnt;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    load_state<NTs>(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    __syncthreads();
    phase_metrics<NTs>(sm, SegView{}, nullptr, nullptr, nullptr, N, true, false, 0.f, cnt);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += NTs)
        if (sm.valid[i]) A.m.ov[a0 + i] = merged_ov(sm, i);
    publish_counts(sm, A, cnt);
}

__global__ void __launch_bounds__(NTs) k_plain_offroad(const StepArgs A, int s) {
    __shared__ AgentSmem sm;
    init_cta(sm);
    Counts cnt;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    load_state<NTs>(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    __syncthreads();
    phase_metrics<NTs>(sm, global_view(A.segs, s), A.hint ? A.hint + 4 * a0 : nullptr,
                       A.tlist ? A.tlist + kList * a0 : nullptr, A.tmeta ? A.tmeta + a0 : nullptr, N, false, true,
                       kListLook * A.p.dt, cnt);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += NTs)
        if (sm.valid[i]) A.m.off[a0 + i] = sm.off[i];
    publish_counts(sm, A, cnt);
}

__global__ void __launch_bounds__(NTs) k_plain_finish(const StepArgs A, int s) {
    __shared__ AgentSmem sm;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    load_state<NTs>(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    for (int i = threadIdx.x; i < N; i += NTs) {
        const int g = a0 + i;
        sm.ovk[i] = ukey(A.m.ov[g]);
        sm.off[i] = A.m.off[g];
        if (A.do_transition && sm.valid[i])  // transition A.in -> A.out
            sm.kin[i] = kin_infeasible(A.p, A.in.vx[g], A.in.vy[g], A.in.th[g], A.in.th_lo[g], sm.vx[i], sm.vy[i]);
    }
    __syncthreads();
    phase_finish<NTs>(sm, A, A.m, A.m.reward + s, A.t_log, a0, N);
}

// ---------------------------------------------------------------------------
// Expert actions, open loop (Sec. 5.2): element (k, g) is the inverse of
// agent g's action space (App. A.1) from log row t0+k to row t0+k+1.  A
// thread takes one agent and a chunk of kExpertChunk steps: it loads the
// chunk's kExpertChunk+1 log rows of that agent first (all loads in flight
// together), then writes the chunk's actions.  The bicycle inverse (atan2,
// square roots, quotients) keeps the kernel issue-bound; chunks of 4 (more
// warps in flight, fewer registers) measured faster than 2 or 8, than the
// chunk index fastest in the grid, and than a rolling window of prefetched
// rows that reads each row once.  Consecutive threads take
// consecutive agents, so every load and store of a warp is one coalesced row
// segment.  HBM-bound: per policy agent-step 12 B of log read (heading and
// velocity for bicycle agents, position and heading for delta agents), per
// agent-step 12 B of action written; the first row of a chunk is read twice.
// ---------------------------------------------------------------------------
constexpr int kExpertChunk = 4;

// 8 CTAs per SM (32 registers): all 64 warps in flight, 4 % faster than the
// 38-register build at 6 CTAs.
__global__ void __launch_bounds__(256, 8) k_expert_actions(const StepArgs A, int t0, int T, float* __restrict__ act) {
    const int g = blockIdx.x * 256 + threadIdx.x;
    if (g >= A.N_tot) return;
    const size_t n = static_cast<size_t>(A.N_tot);
    const int k0 = blockIdx.y * kExpertChunk;
    const int m = min(kExpertChunk, T - k0);  // steps of this chunk
    const int kind = A.valid[g] ? A.kind[g] : -1;
    const bool bic = kind == WSIM_KIND_BICYCLE, del = kind == WSIM_KIND_DELTA;
    // Three logged quantities per row: bicycle (vx, vy, heading), delta (x, y, heading).
    const float* __restrict__ q0 = bic ? A.log_vx : A.log_x;
    const float* __restrict__ q1 = bic ? A.log_vy : A.log_y;
    const float* __restrict__ q2 = A.log_th;
    float r0[kExpertChunk + 1], r1[kExpertChunk + 1], r2[kExpertChunk + 1];
    if (bic || del) {
        const size_t base = (static_cast<size_t>(t0) + k0) * n + g;
#pragma unroll
        for (int j = 0; j <= kExpertChunk; ++j) {
            if (j <= m) {
                r0[j] = q0[base + j * n];
                r1[j] = q1[base + j * n];
                r2[j] = q2[base + j * n];
            }
        }
    }
    // speed of each logged row, once (each serves two consecutive actions)
    float sp[kExpertChunk + 1];
#pragma unroll
    for (int j = 0; j <= kExpertChunk; ++j) sp[j] = (bic && j <= m) ? sqrtf(fmaf(r0[j], r0[j], r1[j] * r1[j])) : 0.f;
    float* out = act + static_cast<size_t>(k0) * 3 * n + g;
#pragma unroll
    for (int j = 0; j < kExpertChunk; ++j) {
        if (j < m) {
            float u0 = 0.f, u1 = 0.f, u2 = 0.f;
            if (bic) {
                const BicycleInv r = bicycle_inverse_v(A.p, sp[j], sp[j + 1], r2[j], 0.f, r0[j + 1], r1[j + 1]);
                u0 = r.a;
                u1 = r.kappa;
            } else if (del) {
                u0 = r0[j + 1] - r0[j];
                u1 = r1[j + 1] - r1[j];
                u2 = r2[j + 1] - r2[j];
            }
            out[0] = u0;
            out[n] = u1;
            out[2 * n] = u2;
            out += 3 * n;
        }
    }
}

cudaError_t launch_expert_actions(const StepArgs& a, int t0, int T, float* act, cudaStream_t st) {
    if (T == 0 || a.N_tot == 0) return cudaSuccess;
    const dim3 grid((a.N_tot + 255) / 256, (T + kExpertChunk - 1) / kExpertChunk);
    k_expert_actions<<<grid, 256, 0, st>>>(a, t0, T, act);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Discrete actions (Sec. 5.2): one thread per agent-step, agents fastest.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_discretize(const StepArgs A, const float* act, int T, int32_t* idx) {
    const size_t n_tot = static_cast<size_t>(A.N_tot), n = static_cast<size_t>(T) * n_tot;
    for (size_t q = static_cast<size_t>(blockIdx.x) * 256 + threadIdx.x; q < n; q += static_cast<size_t>(gridDim.x) * 256) {
        const size_t k = q / n_tot, g = q - k * n_tot;
        const float* u = act + k * 3 * n_tot + g;
        idx[q] = A.valid[g] ? disc_encode(A.p, A.kind[g], u[0], u[n_tot], u[2 * n_tot]) : -1;
    }
}

__global__ void __launch_bounds__(256) k_decode_actions(const StepArgs A, const int32_t* idx, int T, float* act) {
    const size_t n_tot = static_cast<size_t>(A.N_tot), n = static_cast<size_t>(T) * n_tot;
    for (size_t q = static_cast<size_t>(blockIdx.x) * 256 + threadIdx.x; q < n; q += static_cast<size_t>(gridDim.x) * 256) {
        const size_t k = q / n_tot, g = q - k * n_tot;
        float u0, u1, u2;
        if (!disc_decode(A.p, A.kind[g], idx[q], u0, u1, u2)) set_status(A.status, WSIM_EINVAL);
        float* o = act + k * 3 * n_tot + g;
        o[0] = u0;
        o[n_tot] = u1;
        o[2 * n_tot] = u2;
    }
}

static int grid_for(size_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t blocks = (n + 255) / 256;
    return static_cast<int>(blocks < static_cast<size_t>(sms) * 8 ? blocks : static_cast<size_t>(sms) * 8);
}

cudaError_t launch_discretize(const StepArgs& a, const float* act, int T, int32_t* idx, cudaStream_t st) {
    const size_t n = static_cast<size_t>(T) * static_cast<size_t>(a.N_tot);
    if (n == 0) return cudaSuccess;
    k_discretize<<<grid_for(n), 256, 0, st>>>(a, act, T, idx);
    return cudaGetLastError();
}

cudaError_t launch_decode_actions(const StepArgs& a, const int32_t* idx, int T, float* act, cudaStream_t st) {
    const size_t n = static_cast<size_t>(T) * static_cast<size_t>(a.N_tot);
    if (n == 0) return cudaSuccess;
    k_decode_actions<<<grid_for(n), 256, 0, st>>>(a, idx, T, act);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Road-edge segment packing (wsim_init).
// ---------------------------------------------------------------------------
struct RgView {
    const float *x, *y;
    const int32_t* poly;
    const uint8_t *type, *valid;
};

__device__ __forceinline__ bool is_seg(const RgView& r, int r0, int r1, int k) {
    if (k < r0 || k + 1 >= r1) return false;
    return r.valid[k] && r.valid[k + 1] && r.type[k] == WSIM_RG_EDGE && r.type[k + 1] == WSIM_RG_EDGE &&
           r.poly[k] == r.poly[k + 1];
}

// Packing order of one scene's road-edge segments: roadgraph order, with
// every run of consecutive segments (one polyline without a gap) starting on
// a kTile boundary, so that no culling tile holds two runs (a tile across two
// polylines would have a capsule as long as the distance between them).
// One warp per scene, 32 points per iteration; emit(k, p) receives segment
// k's scene-relative position p, pad(p) each padding position.  Returns the
// number of positions used (padding between runs included).
__device__ __forceinline__ unsigned lanes_between(int a, int b) {  // bits [a, b)
    const unsigned hi = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
    return hi & ~((1u << a) - 1u);
}

template <class Emit, class Pad>
__device__ int pack_runs(const RgView& rg, int r0, int r1, int lane, Emit emit, Pad pad) {
    int pos = 0;  // next free position
    for (int c0 = r0; c0 < r1; c0 += 32) {
        const int k = c0 + lane;
        const bool f = is_seg(rg, r0, r1, k);
        const bool st = f && !is_seg(rg, r0, r1, k - 1);
        const unsigned fm = __ballot_sync(kFull, f);
        unsigned starts = __ballot_sync(kFull, st);
        int cur = pos, prev = 0, base = pos, first = 0;  // lanes before the first start continue a run
        while (starts) {
            const int s = __ffs(starts) - 1;
            starts &= starts - 1;
            cur += __popc(fm & lanes_between(prev, s));
            const int aligned = (cur + kTile - 1) / kTile * kTile;
            if (lane < aligned - cur) pad(cur + lane);
            cur = aligned;
            if (lane >= s) {
                base = cur;
                first = s;
            }
            prev = s;
        }
        cur += __popc(fm & lanes_between(prev, 32));
        if (f) emit(k, base + (lane - first));
        pos = cur;
    }
    return pos;
}

__global__ void __launch_bounds__(32) k_seg_count(const int32_t* rg_off, RgView rg, int32_t* cnt) {
    const int s = blockIdx.x;
    const int n = pack_runs(rg, rg_off[s], rg_off[s + 1], threadIdx.x, [](int, int) {}, [](int) {});
    if (threadIdx.x == 0) cnt[s] = n;
}

// Far-away padding segment: its squared distance overflows to +inf, so it
// never wins a nearest-segment search; flags 0 (not a segment).
constexpr float kFarAway = 1e30f;

__global__ void __launch_bounds__(32) k_seg_pack(const int32_t* rg_off, RgView rg, const int32_t* seg_off,
                                                 float4* geo, float* inv, uint8_t* flags) {
    const int s = blockIdx.x;
    const int r0 = rg_off[s], r1 = rg_off[s + 1];
    const int e0 = seg_off[s];
    const int n = pack_runs(
        rg, r0, r1, threadIdx.x,
        [&](int k, int p) {
            const float ax = rg.x[k], ay = rg.y[k];
            const float ux = rg.x[k + 1] - ax, uy = rg.y[k + 1] - ay;
            geo[e0 + p] = make_float4(ax, ay, ux, uy);
            inv[e0 + p] = 1.0f / fmaf(ux, ux, uy * uy);
            flags[e0 + p] = (is_seg(rg, r0, r1, k - 1) ? 1 : 0) | (is_seg(rg, r0, r1, k + 1) ? 2 : 0) | 4;
        },
        [&](int p) {
            geo[e0 + p] = make_float4(kFarAway, kFarAway, 0.f, 0.f);
            inv[e0 + p] = 0.f;
            flags[e0 + p] = 0;
        });
    // the scene's tail up to its aligned end
    const int end = (n + kSegAlign - 1) / kSegAlign * kSegAlign;
    for (int p = n + static_cast<int>(threadIdx.x); p < end; p += 32) {
        geo[e0 + p] = make_float4(kFarAway, kFarAway, 0.f, 0.f);
        inv[e0 + p] = 0.f;
        flags[e0 + p] = 0;
    }
}

// Per tile: a capsule around its segments: the chord from the first
// segment's start to the last segment's end, and the largest distance of any
// segment end point from that chord (rounded up).  Record 0: (start, chord);
// record 1: (radius, 1/|chord|^2, 0, 0).  Both chord ends lie on segments.
// A tile holds one run: segments first, then padding (flags 0).
__global__ void __launch_bounds__(256) k_tile_build(const int32_t* seg_off, const int32_t* seg_cnt,
                                                    const float4* geo, const uint8_t* flags, float4* tiles) {
    const int s = blockIdx.x;
    const int e0 = seg_off[s], E = seg_cnt[s];
    const int nt = (E + kTile - 1) / kTile;
    for (int t = threadIdx.x; t < nt; t += 256) {
        const int b = e0 + t * kTile;
        int n = min(kTile, E - t * kTile);
        while (n > 1 && !(flags[b + n - 1] & 4)) --n;
        const float4 A = geo[b], Z = geo[b + n - 1];
        const float sx = A.x, sy = A.y;
        const float dx = (Z.x + Z.z) - sx, dy = (Z.y + Z.w) - sy;
        const float dd = fmaf(dx, dx, dy * dy);
        const float inv = dd > 0.f ? 1.0f / dd : 0.f;
        float r2 = 0.f;
        for (int j = 0; j < n; ++j) {
            const float4 G = geo[b + j];
            for (int end = 0; end < 2; ++end) {
                const float wx = (end ? G.x + G.z : G.x) - sx, wy = (end ? G.y + G.w : G.y) - sy;
                const float u = __saturatef(fmaf(wx, dx, wy * dy) * inv);
                const float ex = fmaf(-u, dx, wx), ey = fmaf(-u, dy, wy);
                r2 = fmaxf(r2, fmaf(ex, ex, ey * ey));
            }
        }
        const size_t ti = static_cast<size_t>(e0 / kTile + t);
        tiles[2 * ti] = make_float4(sx, sy, dx, dy);
        tiles[2 * ti + 1] = make_float4(sqrtf(r2) * 1.00001f + 1e-4f, inv, 0.f, 0.f);
    }
}

// Super-tile order of one scene's tiles: the tiles sorted by the Morton code
// of their chord midpoints (8 bits per axis over the scene's extent; ties by
// tile index, so the order is unique), one CTA per scene, bitonic sort of
// (code << 16 | tile) keys in shared memory.  Consecutive tiles in this
// order lie close together, so kSuper of them make a compact super-tile
// whatever the roadgraph's polyline order is.
__device__ __forceinline__ uint32_t spread8(uint32_t v) {  // bits 0..7 -> even bits 0..14
    v &= 0xffu;
    v = (v | (v << 4)) & 0x0f0fu;
    v = (v | (v << 2)) & 0x3333u;
    v = (v | (v << 1)) & 0x5555u;
    return v;
}

constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const int32_t* seg_off, const int32_t* seg_cnt,
                                                              const float4* tiles, uint16_t* tperm) {
    __shared__ uint32_t key[kOrderMaxTiles];
    __shared__ float red[4][kOrderThreads / 32];
    const int s = blockIdx.x;
    const int e0 = seg_off[s], E = seg_cnt[s];
    const int nt = (E + kTile - 1) / kTile;
    const size_t tb = static_cast<size_t>(e0 / kTile);
    if (nt > kOrderMaxTiles) {  // identity
        for (int t = threadIdx.x; t < nt; t += kOrderThreads) tperm[tb + t] = static_cast<uint16_t>(t);
        return;
    }
    // extent of the chord midpoints (fminf / fmaxf ignore NaN)
    float lo_x = WSIM_INF, lo_y = WSIM_INF, hi_x = -WSIM_INF, hi_y = -WSIM_INF;
    for (int t = threadIdx.x; t < nt; t += kOrderThreads) {
        const float4 C = tiles[2 * (tb + t)];
        const float mx = fmaf(0.5f, C.z, C.x), my = fmaf(0.5f, C.w, C.y);
        lo_x = fminf(lo_x, mx);
        lo_y = fminf(lo_y, my);
        hi_x = fmaxf(hi_x, mx);
        hi_y = fmaxf(hi_y, my);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = lo_x;
        red[1][warp] = lo_y;
        red[2][warp] = hi_x;
        red[3][warp] = hi_y;
    }
    __syncthreads();
    lo_x = lo_y = WSIM_INF;
    hi_x = hi_y = -WSIM_INF;
    for (int w = 0; w < kOrderThreads / 32; ++w) {
        lo_x = fminf(lo_x, red[0][w]);
        lo_y = fminf(lo_y, red[1][w]);
        hi_x = fmaxf(hi_x, red[2][w]);
        hi_y = fmaxf(hi_y, red[3][w]);
    }
    const float sx = hi_x > lo_x ? 255.f / (hi_x - lo_x) : 0.f;
    const float sy = hi_y > lo_y ? 255.f / (hi_y - lo_y) : 0.f;
    int n2 = 1;
    while (n2 < nt) n2 <<= 1;
    for (int t = threadIdx.x; t < n2; t += kOrderThreads) {
        uint32_t k = 0xffffffffu;  // padding sorts last
        if (t < nt) {
            const float4 C = tiles[2 * (tb + t)];
            const float mx = fmaf(0.5f, C.z, C.x), my = fmaf(0.5f, C.w, C.y);
            // clamped cell coordinates (a NaN or infinite extent gives cell 0)
            const uint32_t qx = static_cast<uint32_t>(fminf(255.f, fmaxf(0.f, (mx - lo_x) * sx)));
            const uint32_t qy = static_cast<uint32_t>(fminf(255.f, fmaxf(0.f, (my - lo_y) * sy)));
            k = ((spread8(qx) | (spread8(qy) << 1)) << 16) | static_cast<uint32_t>(t);
        }
        key[t] = k;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += kOrderThreads) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t a = key[i], b = key[l];
                    if (((i & k) == 0) == (a > b)) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < nt; t += kOrderThreads) tperm[tb + t] = static_cast<uint16_t>(key[t] & 0xffffu);
}

// Per super-tile: bounding box of the capsules of its kSuper tiles (in
// super-tile order).
__global__ void __launch_bounds__(256) k_super_build(const int32_t* seg_off, const int32_t* seg_cnt,
                                                     const int32_t* soff, const float4* tiles,
                                                     const uint16_t* tperm, float4* sup) {
    const int s = blockIdx.x;
    const int e0 = seg_off[s], E = seg_cnt[s];
    const int nt = (E + kTile - 1) / kTile;
    const int ns = (nt + kSuper - 1) / kSuper;
    for (int j = threadIdx.x; j < ns; j += 256) {
        float x0 = WSIM_INF, y0 = WSIM_INF, x1 = -WSIM_INF, y1 = -WSIM_INF;
        for (int q = j * kSuper; q < min(nt, (j + 1) * kSuper); ++q) {
            const int t = tperm ? tperm[e0 / kTile + q] : q;
            const size_t ti = static_cast<size_t>(e0 / kTile) + t;
            const float4 C = tiles[2 * ti];
            const float r = tiles[2 * ti + 1].x;
            x0 = fminf(x0, fminf(C.x, C.x + C.z) - r);
            y0 = fminf(y0, fminf(C.y, C.y + C.w) - r);
            x1 = fmaxf(x1, fmaxf(C.x, C.x + C.z) + r);
            y1 = fmaxf(y1, fmaxf(C.y, C.y + C.w) + r);
        }
        sup[soff[s] + j] = make_float4(x0, y0, x1, y1);
    }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_seg_count(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                             const uint8_t* rg_type, const uint8_t* rg_valid, int S, int32_t* cnt,
                             cudaStream_t st) {
    RgView rg{rg_x, rg_y, rg_poly, rg_type, rg_valid};
    k_seg_count<<<S, 32, 0, st>>>(rg_off, rg, cnt);
    return cudaGetLastError();
}

cudaError_t launch_seg_pack(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                            const uint8_t* rg_type, const uint8_t* rg_valid, int S, const int32_t* seg_off,
                            float4* geo, float* inv, uint8_t* flags, cudaStream_t st) {
    RgView rg{rg_x, rg_y, rg_poly, rg_type, rg_valid};
    k_seg_pack<<<S, 32, 0, st>>>(rg_off, rg, seg_off, geo, inv, flags);
    return cudaGetLastError();
}

cudaError_t launch_tile_build(int S, const int32_t* seg_off, const int32_t* seg_cnt, const float4* geo,
                              const uint8_t* flags, float4* tiles, cudaStream_t st) {
    k_tile_build<<<S, 256, 0, st>>>(seg_off, seg_cnt, geo, flags, tiles);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(int S, const int32_t* seg_off, const int32_t* seg_cnt, const float4* tiles,
                              uint16_t* tperm, cudaStream_t st) {
    k_tile_order<<<S, kOrderThreads, 0, st>>>(seg_off, seg_cnt, tiles, tperm);
    return cudaGetLastError();
}

cudaError_t launch_super_build(int S, const int32_t* seg_off, const int32_t* seg_cnt, const int32_t* soff,
                               const float4* tiles, const uint16_t* tperm, float4* sup, cudaStream_t st) {
    k_super_build<<<S, 256, 0, st>>>(seg_off, seg_cnt, soff, tiles, tperm, sup);
    return cudaGetLastError();
}

// Largest route-point spacing per route parameter, one thread per agent: a
// sample moves at most rf metres per metre of route parameter, so samples
// k dq apart lie within k dq rf of each other (the IDM lead search's group
// circles).
__global__ void __launch_bounds__(256) k_route_speed(const int32_t* route_off, const float* rx, const float* ry,
                                                     int N, float inv_h, float* rf) {
    const int g = blockIdx.x * 256 + threadIdx.x;
    if (g >= N) return;
    float m = 0.f;
    for (int k = route_off[g]; k + 1 < route_off[g + 1]; ++k) {
        const float d = hypotf(rx[k + 1] - rx[k], ry[k + 1] - ry[k]);
        m = d < WSIM_INF ? fmaxf(m, d) : WSIM_INF;  // NaN or inf: no bound
    }
    rf[g] = m < WSIM_INF ? m * inv_h * 1.00001f : WSIM_INF;
}

cudaError_t launch_route_speed(const int32_t* route_off, const float* rx, const float* ry, int N, float inv_h,
                               float* rf, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    k_route_speed<<<(N + 255) / 256, 256, 0, st>>>(route_off, rx, ry, N, inv_h, rf);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t st) {
    if (a.count)
        k_step<true><<<grid, NTs, 0, st>>>(a);
    else
        k_step<false><<<grid, NTs, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plain_scene(const StepArgs& a, int scene, cudaStream_t st) {
    if (a.do_transition) k_plain_transition<<<1, NTs, 0, st>>>(a, scene);
    if (a.do_metrics) {
        k_plain_overlap<<<1, NTs, 0, st>>>(a, scene);
        k_plain_offroad<<<1, NTs, 0, st>>>(a, scene);
        k_plain_finish<<<1, NTs, 0, st>>>(a, scene);
    }
    return cudaGetLastError();
}

int step_blocks_per_sm() {
    int n = 0;
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<false>, NTs, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_step<true>, NTs, 0) != cudaSuccess)
        return 1;
    n = m < n ? m : n;
    return n > 0 ? n : 1;
}

}  // namespace wsim
