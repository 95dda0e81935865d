// Backpropagation through whole rollouts (sm_103a): the differentiable
// simulation the paper names as future work (Sec. 6), with the loss
//     L = sum_t sum_i d_i(t)^2 + lambda sum_t sum_{i<j} tau softplus(d_ij(t)/tau)
// over valid agents, d_i the log divergence (Sec. 3.4) and d_ij the SAT
// overlap depth (Sec. 3.4 collision), differentiated with respect to every
// action of the bicycle and delta agents (App. A.1).  IDM agents (Sec. 3.5)
// move as in the forward simulation and are constants for differentiation.
//
// One CTA owns a scene for the whole computation.  Forward: T steps with the
// shared step phases, the loss summed in a fixed order, and the state stored
// every `ck` steps (and at T).  Backward: segments from last to first; each
// recomputes its inner states from its checkpoint with the same code (so
// ck = 10 and ck = 1 give bit-identical results), then runs the reverse
// sweep: the adjoint of the loss at t+1 (each pair evaluated once; the terms
// summed in a fixed order through per-warp buffers: no float atomics) and
// the adjoint of the transition t -> t+1, which yields dL/d(actions at t).
#include <cstring>

#include "wsim_phases.cuh"

namespace wsim {

constexpr int NTb = 512;  // 16 warps per scene: the pair loops take N / 16 agents per warp
constexpr int NWb = NTb / 32;

struct BpttArgs {
    StepArgs A;      // batch, actions (act = [T][3][N_tot]), in = state t0, t_log = t0 + 1, T
    float* ckpt;     // [n_ckpt][10][N_tot]
    float* segbuf;   // [ck + 1][10][N_tot]
    int ck;
    double* loss;    // [S] (may be null in the recording forward)
    float* dact;     // [T][3][N_tot] (may be null)
    float lambda, tau;
    int scene;       // >= 0: this scene only (plain path); -1: persistent over the work list
    // Recording forward and the backward of a weighted objective.
    int metrics;                           // recording forward: metric rows (A.m) and records
    int16_t* rec_ov;                       // [T][N_tot] partner of the deepest overlap (-1: none)
    int32_t* rec_off;                      // [T][N_tot] off-road record (offroad_code, -1: none)
    const float *g_logdiv, *g_ov, *g_off;  // [T][N_tot] weights of the metric rows (may be null)
    const double* loss_w;                  // [S] weight of each scene's loss (null: 1)
    StateP dst0;                           // dL/d(state t0) (x == nullptr: not wanted)
};

struct AdjSmem {
    float x[kMaxN], y[kMaxN], th[kMaxN], vx[kMaxN], vy[kMaxN];
    float part[kMaxN];
    float cx[kMaxN], cy[kMaxN], cth[kMaxN];  // an agent's overlap term, partner's share
    float lx[kMaxN], ly[kMaxN];              // the current step's logged positions
    int16_t pidx[kMaxN];                     // ... and the partner (-1: none)
    uint8_t pli[NWb][kMaxN + 32], plj[NWb][kMaxN + 32];  // each warp's pending pairs (PairQueue)
    double total;
};

// The logged positions of log row t_log into adj.lx / adj.ly (thread per
// agent, in a per-agent phase): the loss and its adjoint read them in their
// pair loops, one parallel round trip to memory per step.
__device__ __forceinline__ void load_log_row(AdjSmem& adj, const StepArgs& A, int a0, int N, int t_log) {
    const size_t row = static_cast<size_t>(t_log) * A.N_tot + a0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        adj.lx[i] = A.log_x[row + i];
        adj.ly[i] = A.log_y[row + i];
    }
}

__device__ __forceinline__ StateP slot_state(float* base, int slot, int N_tot) {
    float* p = base + static_cast<size_t>(slot) * 10 * N_tot;
    const size_t n = static_cast<size_t>(N_tot);
    return StateP{p, p + n, p + 2 * n, p + 3 * n, p + 4 * n, p + 5 * n, p + 6 * n, p + 7 * n, p + 8 * n, p + 9 * n};
}
__device__ __forceinline__ CStateP cslot(float* base, int slot, int N_tot) {
    const StateP s = slot_state(base, slot, N_tot);
    return CStateP{s.x, s.y, s.x_lo, s.y_lo, s.th, s.th_lo, s.vx, s.vy, s.s, s.s_lo};
}

__device__ __forceinline__ float softplus_f(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }
__device__ __forceinline__ float sigmoid_f(float x) {
    if (x >= 0.f) return 1.f / (1.f + expf(-x));
    const float e = expf(x);
    return e / (1.f + e);
}

// SAT depth of boxes A, B with the partial derivatives of the active
// (first minimal) axis term w.r.t. theta_A, theta_B and d = c_B - c_A.
struct SatGrad {
    float d, dthA, dthB, ddx, ddy;
};

__device__ __forceinline__ SatGrad sat_grad(float dx, float dy, float cA, float sA, float hlA, float hwA, float cB,
                                            float sB, float hlB, float hwB) {
    const float C = fmaf(cA, cB, sA * sB);
    const float S = fmaf(cA, sB, -sA * cB);
    const float aC = fabsf(C), aS = fabsf(S);
    const float sC = C < 0.f ? -1.f : 1.f, sS = S < 0.f ? -1.f : 1.f;
    const float pA = fmaf(dx, cA, dy * sA), qA = fmaf(-dx, sA, dy * cA);
    const float pB = fmaf(dx, cB, dy * sB), qB = fmaf(-dx, sB, dy * cB);
    const float o0 = hlA + fmaf(hlB, aC, hwB * aS) - fabsf(pA);
    const float o1 = hwA + fmaf(hlB, aS, hwB * aC) - fabsf(qA);
    const float o2 = hlB + fmaf(hlA, aC, hwA * aS) - fabsf(pB);
    const float o3 = hwB + fmaf(hlA, aS, hwA * aC) - fabsf(qB);
    int k = 0;
    float m = o0;
    if (o1 < m) { m = o1; k = 1; }
    if (o2 < m) { m = o2; k = 2; }
    if (o3 < m) { m = o3; k = 3; }
    SatGrad g;
    g.d = m;
    if (k == 0) {
        const float sp = pA < 0.f ? -1.f : 1.f;
        g.dthA = hlB * sC * S - hwB * sS * C - sp * qA;
        g.dthB = -hlB * sC * S + hwB * sS * C;
        g.ddx = -sp * cA;
        g.ddy = -sp * sA;
    } else if (k == 1) {
        const float sq = qA < 0.f ? -1.f : 1.f;
        g.dthA = -hlB * sS * C + hwB * sC * S + sq * pA;
        g.dthB = hlB * sS * C - hwB * sC * S;
        g.ddx = sq * sA;
        g.ddy = -sq * cA;
    } else if (k == 2) {
        const float sp = pB < 0.f ? -1.f : 1.f;
        g.dthA = hlA * sC * S - hwA * sS * C;
        g.dthB = -hlA * sC * S + hwA * sS * C - sp * qB;
        g.ddx = -sp * cB;
        g.ddy = -sp * sB;
    } else {
        const float sq = qB < 0.f ? -1.f : 1.f;
        g.dthA = -hlA * sS * C + hwA * sC * S;
        g.dthB = hlA * sS * C - hwA * sC * S + sq * pB;
        g.ddx = sq * sB;
        g.ddy = -sq * cB;
    }
    return g;
}

// Pairs that add exactly nothing: softplus(d/tau) and sigmoid(d/tau) are 0
// in float32 once d/tau < -104 (e^(d/tau) underflows), so a pair whose SAT
// depth bound R_i + R_j - |c_j - c_i| / sqrt(2) (the overlap culling bound)
// lies below -120 tau contributes 0 to the loss and to its gradient and is
// not evaluated.  cut = 120 tau, or -1 (no culling) unless 0 < tau < inf;
// the 1 cm and relative slack cover the float32 centres (high words).
__device__ __forceinline__ float pair_cut(float tau) { return (tau > 0.f && tau < WSIM_INF) ? 120.f * tau : -1.f; }
__device__ __forceinline__ bool pair_far(const AgentSmem& sm, int i, int j, float cut) {
    const float dx = sm.xh[j] - sm.xh[i], dy = sm.yh[j] - sm.yh[i];
    // R_i + R_j with R = hl + hw rounded up
    const float rr = (sm.hl[i] + sm.hw[i] + sm.hl[j] + sm.hw[j]) * 1.000001f + 1e-3f;
    const float r = rr + cut + 0.01f + 1e-6f * (fabsf(sm.xh[i]) + fabsf(sm.yh[i]) + fabsf(sm.xh[j]) + fabsf(sm.yh[j]));
    return cut > 0.f && fmaf(dx, dx, dy * dy) > 2.f * r * r;
}

// A warp's pending pairs (i, j), j > i, in row order and increasing j within
// a row: the valid partners that pair_far does not rule out of each of the
// warp's rows, appended row by row and evaluated 32 at a time, so that the
// pair loops run over full lanes however few partners a row has.  At most
// 31 pairs wait when a row is appended, so kMaxN + 32 entries hold them.
struct PairQueue {
    uint8_t* pi;
    uint8_t* pj;
    int n;
};

__device__ __forceinline__ void append_row(const AgentSmem& sm, int N, int i, int lane, float cut, PairQueue& q,
                                           Counts& cnt) {
    const int n0 = q.n;
    for (int jb = i + 1; jb < N; jb += 32) {
        const int j = jb + lane;
        const bool keep = j < N && sm.valid[j] && !pair_far(sm, i, j, cut);
        const unsigned m = __ballot_sync(kFull, keep);
        if (keep) {
            const int k = q.n + __popc(m & ((1u << lane) - 1u));
            q.pi[k] = static_cast<uint8_t>(i);
            q.pj[k] = static_cast<uint8_t>(j);
        }
        q.n += __popc(m);
    }
    if (lane == 0) cnt.pairs += 2 * (q.n - n0);  // SAT evaluations, two per pair as in the overlap rows
    __syncwarp();
}

// Drops the first 32 pairs (after they were evaluated).
__device__ __forceinline__ void pop32(PairQueue& q, int lane) {
    for (int k = lane; k < q.n - 32; k += 32) {  // lane l moves entries l + 32 c in increasing c
        q.pi[k] = q.pi[k + 32];
        q.pj[k] = q.pj[k + 32];
    }
    q.n -= 32;
    __syncwarp();
}

// Sum of v over the lanes of one row's run [k0, k1) of a batch (fixed
// shuffle tree; lanes outside the run give 0); the run ends at *k1.
__device__ __forceinline__ float run_sum(float v, bool in_run) {
    v = in_run ? v : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Loss terms of the current state (warp per row, rows warp, warp + NWb, ...):
// adj.part[i] = d_i^2 plus the penalty of i's pairs with j > i, the pairs
// evaluated in batches of 32 of the warp's queue and each batch's share of
// a row added to adj.part[i] by one row-run sum (a fixed order).
__device__ void loss_rows_warp(const AgentSmem& sm, AdjSmem& adj, int N, int lane, int warp, float lambda, float tau,
                               Counts& cnt) {
    PairQueue q{adj.pli[warp], adj.plj[warp], 0};
    const float cut = pair_cut(tau);
    auto flush = [&](int m) {
        const int k = lane < m ? lane : 0;
        const int i = q.pi[k], j = q.pj[k];
        float term = 0.f;
        if (lane < m) {
            const float dx = comp_diff(sm.xh[j], sm.xl[j], sm.xh[i], sm.xl[i]);
            const float dy = comp_diff(sm.yh[j], sm.yl[j], sm.yh[i], sm.yl[i]);
            const float d = sat_depth(dx, dy, sm.c[i], sm.s[i], sm.hl[i], sm.hw[i], sm.c[j], sm.s[j], sm.hl[j],
                                      sm.hw[j]);
            term = lambda * tau * softplus_f(d / tau);
        }
        for (int k0 = 0; k0 < m;) {  // one run of equal rows at a time
            const int r = __shfl_sync(kFull, i, k0);
            const unsigned run = __ballot_sync(kFull, lane < m && i == r);
            const float v = run_sum(term, (run >> lane) & 1u);
            if (lane == 0) adj.part[r] += v;
            k0 = 32 - __clz(run);
        }
        __syncwarp();
    };
    for (int i = warp; i < N; i += NWb) {
        if (!sm.valid[i]) {
            if (lane == 0) adj.part[i] = 0.f;
            continue;
        }
        if (lane == 0) {
            const float ex = (sm.xh[i] - adj.lx[i]) + sm.xl[i], ey = (sm.yh[i] - adj.ly[i]) + sm.yl[i];
            adj.part[i] = fmaf(ex, ex, ey * ey);
        }
        append_row(sm, N, i, lane, cut, q, cnt);
        while (q.n >= 32) {
            flush(32);
            pop32(q, lane);
        }
    }
    if (q.n > 0) flush(q.n);
}

// Adds dL/d(x, y, theta) of every valid agent's loss terms at the current
// state (all threads).  Each pair i < j is evaluated once, by the warp that
// owns row i (rows i = warp, warp + NWb, ...): the row agent's terms are
// summed by a warp reduction, the partner's terms go to the warp's buffer
// wbuf[warp] (a warp synchronises between rows), and each agent then sums
// the NWb buffers in warp order.  Fixed order throughout, no float atomics.
constexpr size_t kPairBufFloats = static_cast<size_t>(NWb) * 3 * kMaxN;

// Agent j's per-agent work in the reverse sweep (the column sums closing
// loss_adjoint and the whole of transition_adjoint) runs in thread
// agent_thread(j).  Both loops iterate through this helper, so the thread
// that finishes agent j's sums is the one that reads them next, and the two
// need no barrier in between; load_prev writes only the n* arrays, which
// loss_adjoint does not read.
__device__ __forceinline__ int first_agent() { return threadIdx.x; }
constexpr int kAgentStride = NTb;
static_assert(kAgentStride == NTb, "one agent per thread and stride: the reverse sweep relies on it");

// wl weighs the whole term (the scene's loss weight; 1 gives the loss's own
// gradient bit for bit).
__device__ void loss_adjoint(const AgentSmem& sm, AdjSmem& adj, float* wbuf, int N, int lane, int warp, float lambda,
                             float tau, float wl, Counts& cnt) {
    float* bx = wbuf + static_cast<size_t>(warp) * 3 * kMaxN;
    float* by = bx + kMaxN;
    float* bth = by + kMaxN;
    PairQueue q{adj.pli[warp], adj.plj[warp], 0};
    const float cut = pair_cut(tau);
    for (int j = lane; j < N; j += 32) bx[j] = by[j] = bth[j] = 0.f;
    __syncwarp();
    // A batch of m queued pairs: lane k evaluates pair k; the partner's terms
    // go to the warp's buffer one row run after another (a run's partners
    // are distinct), the row's by a run sum into adj (lane 0).
    auto flush = [&](int m) {
        const int k = lane < m ? lane : 0;
        const int i = q.pi[k], j = q.pj[k];
        float w = 0.f;
        SatGrad G{};
        if (lane < m) {
            const float dx = comp_diff(sm.xh[j], sm.xl[j], sm.xh[i], sm.xl[i]);
            const float dy = comp_diff(sm.yh[j], sm.yl[j], sm.yh[i], sm.yl[i]);
            G = sat_grad(dx, dy, sm.c[i], sm.s[i], sm.hl[i], sm.hw[i], sm.c[j], sm.s[j], sm.hl[j], sm.hw[j]);
            w = lambda * sigmoid_f(G.d / tau);
        }
        for (int k0 = 0; k0 < m;) {
            const int r = __shfl_sync(kFull, i, k0);
            const unsigned run = __ballot_sync(kFull, lane < m && i == r);
            const bool in = (run >> lane) & 1u;
            if (in) {  // j is the second box of the pair
                bx[j] += w * G.ddx;
                by[j] += w * G.ddy;
                bth[j] += w * G.dthB;
            }
            const float gx = run_sum(-w * G.ddx, in), gy = run_sum(-w * G.ddy, in), gth = run_sum(w * G.dthA, in);
            if (lane == 0) {  // i the first
                adj.x[r] += wl * gx;
                adj.y[r] += wl * gy;
                adj.th[r] += wl * gth;
            }
            k0 = 32 - __clz(run);
            __syncwarp();  // the next run may update the same partners
        }
    };
    for (int i = warp; i < N; i += NWb) {
        if (!sm.valid[i]) continue;
        if (lane == 0) {
            const float ex = (sm.xh[i] - adj.lx[i]) + sm.xl[i], ey = (sm.yh[i] - adj.ly[i]) + sm.yl[i];
            adj.x[i] += wl * (2.f * ex);
            adj.y[i] += wl * (2.f * ey);
        }
        append_row(sm, N, i, lane, cut, q, cnt);
        while (q.n >= 32) {
            flush(32);
            pop32(q, lane);
        }
    }
    if (q.n > 0) flush(q.n);
    __syncthreads();
    for (int j = first_agent(); j < N; j += kAgentStride) {  // same mapping as transition_adjoint
        float sx = 0.f, sy = 0.f, st = 0.f;
        for (int w = 0; w < NWb; ++w) {
            const float* b = wbuf + static_cast<size_t>(w) * 3 * kMaxN;
            sx += b[j];
            sy += b[kMaxN + j];
            st += b[2 * kMaxN + j];
        }
        adj.x[j] += wl * sx;
        adj.y[j] += wl * sy;
        adj.th[j] += wl * st;
    }
}

// Adds the derivative of the weighted metric row of the current state
// (metric row t, time t0+t+1) to adj (all threads; agent j's sums in thread
// agent_thread(j)):
//   log divergence d = |p - log|: (p - log) / d;
//   off-road off = +-|corner - q| (q the nearest point of the recorded
//     segment, + off road): +-(corner - q) / |corner - q|, through the
//     corner c + R(theta) (a, b) also into theta;
//   overlap ov_i = d_ij of the recorded partner j: the SAT depth's partial
//     derivatives (active axis) for both agents; the partner's share goes
//     through adj.c* and is summed by the partner's thread in index order.
__device__ void metric_adjoint(const AgentSmem& sm, AdjSmem& adj, const BpttArgs& B, const SegView& V, int t,
                               int a0, int N) {
    const StepArgs& A = B.A;
    const size_t row = static_cast<size_t>(t) * A.N_tot;
    for (int i = first_agent(); i < N; i += kAgentStride) {
        const int g = a0 + i;
        adj.pidx[i] = -1;
        if (!sm.valid[i]) continue;
        float gx = 0.f, gy = 0.f, gth = 0.f;
        const float xih = sm.xh[i], xil = sm.xl[i], yih = sm.yh[i], yil = sm.yl[i];
        const float w_ld = B.g_logdiv ? B.g_logdiv[row + g] : 0.f;
        if (w_ld != 0.f) {
            const float ex = (xih - adj.lx[i]) + xil, ey = (yih - adj.ly[i]) + yil;
            const float ld = sqrtf(fmaf(ex, ex, ey * ey));
            if (ld > 0.f) {
                gx += w_ld * ex / ld;
                gy += w_ld * ey / ld;
            }
        }
        const float w_off = B.g_off ? B.g_off[row + g] : 0.f;
        const int code = w_off != 0.f ? B.rec_off[row + g] : -1;
        if (code >= 0) {
            const int e = code >> 3, k = (code >> 1) & 3;
            const float sgn = (code & 1) ? 1.f : -1.f;
            const float a = (k < 2 ? 1.f : -1.f) * sm.hl[i];
            const float b = (k == 0 || k == 3 ? 1.f : -1.f) * sm.hw[i];
            const float c = sm.c[i], s = sm.s[i];
            const float cl = xil + fmaf(a, c, -b * s), dl = yil + fmaf(a, s, b * c);
            const float4 G = V.geo[e];
            const float wx = (xih - G.x) + cl, wy = (yih - G.y) + dl;
            const float tq = __saturatef(fmaf(wx, G.z, wy * G.w) * V.inv[e]);
            const float ex = fmaf(-tq, G.z, wx), ey = fmaf(-tq, G.w, wy);
            const float d = sqrtf(fmaf(ex, ex, ey * ey));
            if (d > 0.f) {
                const float px = w_off * sgn * ex / d, py = w_off * sgn * ey / d;
                gx += px;
                gy += py;
                gth += px * fmaf(-a, s, -b * c) + py * fmaf(a, c, -b * s);  // d corner / d theta
            }
        }
        const float w_ov = B.g_ov ? B.g_ov[row + g] : 0.f;
        const int j = w_ov != 0.f ? B.rec_ov[row + g] : -1;
        if (j >= 0) {
            const int ia = min(i, j), ib = max(i, j);
            const float dx = comp_diff(sm.xh[ib], sm.xl[ib], sm.xh[ia], sm.xl[ia]);
            const float dy = comp_diff(sm.yh[ib], sm.yl[ib], sm.yh[ia], sm.yl[ia]);
            const SatGrad G = sat_grad(dx, dy, sm.c[ia], sm.s[ia], sm.hl[ia], sm.hw[ia], sm.c[ib], sm.s[ib],
                                       sm.hl[ib], sm.hw[ib]);
            // d d_ab: -(ddx, ddy) and dthA for a, +(ddx, ddy) and dthB for b
            const float sx = i == ia ? -1.f : 1.f;
            gx += sx * w_ov * G.ddx;
            gy += sx * w_ov * G.ddy;
            gth += w_ov * (i == ia ? G.dthA : G.dthB);
            adj.cx[i] = -sx * w_ov * G.ddx;
            adj.cy[i] = -sx * w_ov * G.ddy;
            adj.cth[i] = w_ov * (i == ia ? G.dthB : G.dthA);
            adj.pidx[i] = static_cast<int16_t>(j);
        }
        adj.x[i] += gx;
        adj.y[i] += gy;
        adj.th[i] += gth;
    }
    __syncthreads();
    for (int j = first_agent(); j < N; j += kAgentStride) {  // same mapping as transition_adjoint
        float sx = 0.f, sy = 0.f, st = 0.f;
        for (int i = 0; i < N; ++i) {
            if (adj.pidx[i] == j) {
                sx += adj.cx[i];
                sy += adj.cy[i];
                st += adj.cth[i];
            }
        }
        adj.x[j] += sx;
        adj.y[j] += sy;
        adj.th[j] += st;
    }
}

// Load state t into the n* arrays (the transition adjoint reads it there).
__device__ void load_prev(AgentSmem& sm, const CStateP& st, int a0, int N) {
    for (int i = threadIdx.x; i < N; i += NTb) {
        const int g = a0 + i;
        sm.nth[i] = st.th[g];
        sm.ntl[i] = st.th_lo[g];
        sm.nvx[i] = st.vx[g];
        sm.nvy[i] = st.vy[g];
    }
}

// Adjoint of the transition t -> t+1 (thread per agent): state t in the n*
// arrays, state t+1 in the current arrays, adj = dL/d(state t+1) on entry
// and dL/d(state t) on exit; writes dL/d(actions at t).
__device__ void transition_adjoint(AgentSmem& sm, AdjSmem& adj, const BpttArgs& B, int t, int a0, int N) {
    const StepArgs& A = B.A;
    const float dt = A.p.dt, hdt2 = 0.5f * dt * dt;
    const float* act = A.act + static_cast<size_t>(t) * 3 * A.N_tot;
    for (int i = first_agent(); i < N; i += kAgentStride) {  // same mapping as loss_adjoint's column sums
        const int g = a0 + i;
        const int kind = sm.kind[i];
        float ga = 0.f, gk = 0.f, g2 = 0.f;
        if (!sm.valid[i]) {
            // held state: the adjoint passes through unchanged
        } else if (kind == WSIM_KIND_IDM) {
            adj.x[i] = adj.y[i] = adj.th[i] = adj.vx[i] = adj.vy[i] = 0.f;  // stop-gradient
        } else if (kind == WSIM_KIND_BICYCLE) {
            const float a = act[g], kap = act[A.N_tot + g];
            const float vx = sm.nvx[i], vy = sm.nvy[i];
            const float v = sqrtf(fmaf(vx, vx, vy * vy));
            float c, s;
            comp_sincos(sm.nth[i], sm.ntl[i], c, s);
            const float cn = sm.c[i], sn = sm.s[i];
            const float vn = fmaf(a, dt, v);
            const float X = adj.x[i], Y = adj.y[i], TH = adj.th[i], VX = adj.vx[i], VY = adj.vy[i];
            const float vbn = fmaf(VX, cn, VY * sn);
            const float thb = TH + vn * fmaf(-VX, sn, VY * cn);
            ga = vbn * dt + thb * kap * hdt2 + hdt2 * fmaf(X, c, Y * s);
            gk = thb * fmaf(v, dt, a * hdt2);
            const float vb = vbn + thb * kap * dt;
            adj.th[i] = thb + a * hdt2 * fmaf(-X, s, Y * c);
            adj.vx[i] = X * dt + (v > 0.f ? vb * vx / v : 0.f);
            adj.vy[i] = Y * dt + (v > 0.f ? vb * vy / v : 0.f);
        } else {  // delta
            const float X = adj.x[i], Y = adj.y[i];
            ga = X + adj.vx[i] / dt;
            gk = Y + adj.vy[i] / dt;
            g2 = adj.th[i];
            adj.vx[i] = adj.vy[i] = 0.f;
        }
        if (B.dact) {
            float* d = B.dact + static_cast<size_t>(t) * 3 * A.N_tot;
            d[g] = ga;
            d[A.N_tot + g] = gk;
            d[2 * static_cast<size_t>(A.N_tot) + g] = g2;
        }
    }
}

// One step's loss of the current state (all threads; the logged positions
// in adj.lx / adj.ly): each warp's rows into adj.part, then (after the
// caller's barrier) warp 0 adds them in a fixed order; see loss_sum.
__device__ __forceinline__ void loss_rows(const AgentSmem& sm, AdjSmem& adj, const BpttArgs& B, int N, Counts& cnt) {
    loss_rows_warp(sm, adj, N, threadIdx.x & 31, threadIdx.x >> 5, B.lambda, B.tau, cnt);
}
// The step's loss in a fixed order: lane-strided sums, then a fixed shuffle tree.
__device__ __forceinline__ void loss_sum(AdjSmem& adj, int N) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        float step = 0.f;
        for (int i = lane; i < N; i += 32) step += adj.part[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) step += __shfl_xor_sync(kFull, step, o);
        if (lane == 0) adj.total += static_cast<double>(step);
    }
}

// Reverse sweep over the checkpointed rollout of scene s: segments from last
// to first, each recomputed from its checkpoint with the forward's code (so
// the checkpoint interval does not change a bit), then, step by step from
// the last, the adjoint of the loss at t+1 weighted by wl (skipped for wl =
// 0), the adjoint of the weighted metric row t (when metric weights are
// given), and the adjoint of the transition t -> t+1, which writes
// dL/d(actions at t).  dL/d(state t0) remains in adj and goes to B.dst0.
__device__ void reverse_sweep(AgentSmem& sm, AdjSmem& adj, float* wbuf, const BpttArgs& B, int s, float wl,
                              Counts& cnt) {
    const StepArgs& A = B.A;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int T = A.T, ck = B.ck;
    const int nseg = (T + ck - 1) / ck;
    const bool metrics = B.g_logdiv || B.g_ov || B.g_off;
    const SegView V = global_view(A.segs, s);
    for (int i = first_agent(); i < N; i += kAgentStride) adj.x[i] = adj.y[i] = adj.th[i] = adj.vx[i] = adj.vy[i] = 0.f;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int a = sg * ck, b = min(a + ck, T);
        // Recompute the inner states a+1 .. b-1 of the segment.
        if (b - a > 1) {
            __syncthreads();
            load_state<NTb>(sm, A, cslot(B.ckpt, sg, A.N_tot), a0, N);
            __syncthreads();
            for (int t = a; t < b - 1; ++t) {
                phase_transition<NTb>(sm, A, A.act + static_cast<size_t>(t) * 3 * A.N_tot, A.t_log + t, a0, N, cnt);
                __syncthreads();
                const StateP o = slot_state(B.segbuf, t + 1 - a, A.N_tot);
                writeback<NTb>(sm, A.p, &o, a0, N);
                __syncthreads();
            }
        }
        for (int t = b - 1; t >= a; --t) {
            __syncthreads();
            // state t+1: the next checkpoint or a recomputed state
            const CStateP nxt = (t + 1 == b) ? cslot(B.ckpt, (b + ck - 1) / ck, A.N_tot)
                                             : cslot(B.segbuf, t + 1 - a, A.N_tot);
            load_state<NTb>(sm, A, nxt, a0, N);
            // state t into the n* arrays, which the loss and metric adjoints do not read
            const CStateP cur = (t == a) ? cslot(B.ckpt, sg, A.N_tot) : cslot(B.segbuf, t - a, A.N_tot);
            load_prev(sm, cur, a0, N);
            load_log_row(adj, A, a0, N, A.t_log + t);
            __syncthreads();
            if (wl != 0.f) loss_adjoint(sm, adj, wbuf, N, lane, warp, B.lambda, B.tau, wl, cnt);
            if (metrics) metric_adjoint(sm, adj, B, V, t, a0, N);
            // both adjoints end with agent j's sums in the thread that takes
            // agent j here: no barrier in between
            transition_adjoint(sm, adj, B, t, a0, N);
        }
    }
    if (B.dst0.x) {
        // x = x_hi + x_lo: both words get dL/dx (likewise theta); the route
        // parameter of IDM agents is a constant
        const StateP& d = B.dst0;
        for (int i = first_agent(); i < N; i += kAgentStride) {
            const int g = a0 + i;
            d.x[g] = d.x_lo[g] = adj.x[i];
            d.y[g] = d.y_lo[g] = adj.y[i];
            d.th[g] = d.th_lo[g] = adj.th[i];
            d.vx[g] = adj.vx[i];
            d.vy[g] = adj.vy[i];
            d.s[g] = d.s_lo[g] = 0.f;
        }
    }
    __syncthreads();
}

// Forward with the loss and checkpoints, then (dact given) the reverse sweep
// of the loss alone.
__device__ void bptt_scene(AgentSmem& sm, AdjSmem& adj, float* wbuf, const BpttArgs& B, int s, Counts& cnt) {
    const StepArgs& A = B.A;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    const int T = A.T, ck = B.ck;

    // Forward.
    load_state<NTb>(sm, A, A.in, a0, N);
    __syncthreads();
    store_state<NTb>(sm, slot_state(B.ckpt, 0, A.N_tot), a0, N);
    if (threadIdx.x == 0) adj.total = 0.0;
    for (int k = 0; k < T; ++k) {
        phase_transition<NTb>(sm, A, A.act + static_cast<size_t>(k) * 3 * A.N_tot, A.t_log + k, a0, N, cnt);
        __syncthreads();
        writeback<NTb>(sm, A.p, nullptr, a0, N);
        load_log_row(adj, A, a0, N, A.t_log + k);
        __syncthreads();
        loss_rows(sm, adj, B, N, cnt);
        if ((k + 1) % ck == 0 || k + 1 == T) store_state<NTb>(sm, slot_state(B.ckpt, (k + 1 + ck - 1) / ck, A.N_tot), a0, N);
        __syncthreads();
        loss_sum(adj, N);
    }
    __syncthreads();
    if (threadIdx.x == 0) B.loss[s] = adj.total;
    if (!B.dact) return;
    reverse_sweep(sm, adj, wbuf, B, s, 1.f, cnt);
}

// Recording forward of scene s: the rollout (every policy agent takes its
// action) with checkpoints every ck steps, the loss (B.loss given) and, with
// B.metrics, every step's metric row (A.m, as wsim_rollout writes it) and
// the records of its deciding indices: the partner of each agent's deepest
// overlap (exact maximum, ties to the lower index) and the corner, segment
// and side of its largest off-road distance (ties to the lower corner).
// tlist / tmeta: the scene's candidate-tile caches of the off-road search.
__device__ void record_scene(AgentSmem& sm, AdjSmem& adj, unsigned long long* k64, uint16_t* tlist, float4* tmeta,
                             const BpttArgs& B, int s) {
    const StepArgs& A = B.A;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    const int lane = threadIdx.x & 31;
    Counts cnt;
    const int T = A.T, ck = B.ck;
    const size_t N_tot = static_cast<size_t>(A.N_tot);
    const SegView V = global_view(A.segs, s);
    load_state<NTb>(sm, A, A.in, a0, N);
    for (int j = threadIdx.x; j < 4 * N; j += NTb) sm.hint[j] = -1;
    for (int j = threadIdx.x; j < N; j += NTb) tmeta[j] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    __syncthreads();
    store_state<NTb>(sm, slot_state(B.ckpt, 0, A.N_tot), a0, N);
    if (threadIdx.x == 0) adj.total = 0.0;
    for (int k = 0; k < T; ++k) {
        phase_transition<NTb>(sm, A, A.act + static_cast<size_t>(k) * 3 * N_tot, A.t_log + k, a0, N, cnt);
        __syncthreads();
        writeback<NTb>(sm, A.p, nullptr, a0, N);
        if (B.loss) load_log_row(adj, A, a0, N, A.t_log + k);
        __syncthreads();
        if (B.metrics) {
            const size_t row = static_cast<size_t>(k) * N_tot;
            overlap_bounds<NTb>(sm, N);
            for (int j = threadIdx.x; j < N; j += NTb) k64[j] = 0ull;
            __syncthreads();
            int32_t* orec = B.rec_off + row + a0;
            for (int q = next_agent(sm, 2, lane); 8 * q < N; q = next_agent(sm, 2, lane))
                offroad_group<true>(sm, V, sm.hint, tlist, tmeta, N, 8 * q, lane, kListLook * A.p.dt, cnt, orec);
            for (int i = next_agent(sm, 1, lane); i < N; i = next_agent(sm, 1, lane))
                if (sm.valid[i]) overlap_row<true>(sm, N, i, lane, cnt, k64);
            __syncthreads();
            const MetricsP m{A.m.ov + row, A.m.off + row, A.m.logdiv + row, A.m.flags + row, nullptr};
            phase_finish<NTb>(sm, A, m, A.m.reward + static_cast<size_t>(k) * A.S + s, A.t_log + k, a0, N);
            for (int i = threadIdx.x; i < N; i += NTb) {
                const bool v = sm.valid[i];
                B.rec_ov[row + a0 + i] = static_cast<int16_t>(v ? argmax_partner(k64[i]) : -1);
                if (!v) orec[i] = -1;
            }
        }
        if (B.loss) loss_rows(sm, adj, B, N, cnt);
        if ((k + 1) % ck == 0 || k + 1 == T) store_state<NTb>(sm, slot_state(B.ckpt, (k + 1 + ck - 1) / ck, A.N_tot), a0, N);
        __syncthreads();
        if (B.loss) loss_sum(adj, N);
    }
    __syncthreads();
    if (B.loss && threadIdx.x == 0) B.loss[s] = adj.total;
    if (A.out.x) store_state<NTb>(sm, A.out, a0, N);
    __syncthreads();
}

// Dynamic shared memory: AgentSmem, AdjSmem, then the pair buffers.
constexpr size_t kAdjOff = (sizeof(AgentSmem) + 15) / 16 * 16;
constexpr size_t kBufOff = (kAdjOff + sizeof(AdjSmem) + 15) / 16 * 16;
constexpr size_t kBpttSmem = kBufOff + kPairBufFloats * sizeof(float);
// Recording forward: AgentSmem, AdjSmem, argmax keys, then the off-road
// candidate-tile caches (list metadata, lists).
constexpr size_t kK64Off = kBufOff;
constexpr size_t kMetaOff = kK64Off + kMaxN * sizeof(unsigned long long);
constexpr size_t kListOff = kMetaOff + kMaxN * sizeof(float4);
constexpr size_t kRecordSmem = kListOff + static_cast<size_t>(kMaxN) * kList * sizeof(uint16_t);

// Next scene of the persistent work list (-1: none left).
__device__ __forceinline__ int next_scene(AgentSmem& sm, const StepArgs& A) {
    if (threadIdx.x == 0) sm.scene = atomicAdd(A.queue, 1);
    __syncthreads();
    const int w = sm.scene;
    return w < A.n_work ? A.order[w] : -1;
}

__global__ void __launch_bounds__(NTb, 2) k_bptt(const BpttArgs B) {
    extern __shared__ __align__(16) unsigned char bdyn[];
    AgentSmem& sm = *reinterpret_cast<AgentSmem*>(bdyn);
    AdjSmem& adj = *reinterpret_cast<AdjSmem*>(bdyn + kAdjOff);
    float* wbuf = reinterpret_cast<float*>(bdyn + kBufOff);
    init_cta(sm);
    Counts cnt;  // published on request (wsim_set_counting): the loss's SAT pair evaluations, the IDM tests
    if (B.scene >= 0) {
        bptt_scene(sm, adj, wbuf, B, B.scene, cnt);
    } else {
        for (int s = next_scene(sm, B.A); s >= 0; s = next_scene(sm, B.A)) {
            bptt_scene(sm, adj, wbuf, B, s, cnt);
            __syncthreads();
        }
    }
    publish_counts(sm, B.A, cnt);
}

__global__ void __launch_bounds__(NTb, 2) k_record(const BpttArgs B) {
    extern __shared__ __align__(16) unsigned char rdyn[];
    AgentSmem& sm = *reinterpret_cast<AgentSmem*>(rdyn);
    AdjSmem& adj = *reinterpret_cast<AdjSmem*>(rdyn + kAdjOff);
    unsigned long long* k64 = reinterpret_cast<unsigned long long*>(rdyn + kK64Off);
    float4* tmeta = reinterpret_cast<float4*>(rdyn + kMetaOff);
    uint16_t* tlist = reinterpret_cast<uint16_t*>(rdyn + kListOff);
    init_cta(sm);
    for (int s = next_scene(sm, B.A); s >= 0; s = next_scene(sm, B.A)) {
        record_scene(sm, adj, k64, tlist, tmeta, B, s);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(NTb, 2) k_backward(const BpttArgs B) {
    extern __shared__ __align__(16) unsigned char bdyn[];
    AgentSmem& sm = *reinterpret_cast<AgentSmem*>(bdyn);
    AdjSmem& adj = *reinterpret_cast<AdjSmem*>(bdyn + kAdjOff);
    float* wbuf = reinterpret_cast<float*>(bdyn + kBufOff);
    init_cta(sm);
    Counts cnt;
    for (int s = next_scene(sm, B.A); s >= 0; s = next_scene(sm, B.A)) {
        reverse_sweep(sm, adj, wbuf, B, s, B.loss_w ? static_cast<float>(B.loss_w[s]) : 0.f, cnt);
        __syncthreads();
    }
    publish_counts(sm, B.A, cnt);
}

static BpttArgs bptt_args(const StepArgs& a, float* ckpt, float* segbuf, int ck, float lambda, float tau) {
    BpttArgs B;
    std::memset(&B, 0, sizeof(B));
    B.A = a;
    B.ckpt = ckpt;
    B.segbuf = segbuf;
    B.ck = ck;
    B.lambda = lambda;
    B.tau = tau;
    B.scene = -1;
    return B;
}

cudaError_t launch_bptt(const StepArgs& a, float* ckpt, float* segbuf, int ck, double* loss, float* dact,
                        float lambda, float tau, int grid, bool plain, cudaStream_t st) {
    BpttArgs B = bptt_args(a, ckpt, segbuf, ck, lambda, tau);
    B.loss = loss;
    B.dact = dact;
    cudaError_t e = cudaFuncSetAttribute(k_bptt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kBpttSmem));
    if (e != cudaSuccess) return e;
    if (plain) {
        for (int s = 0; s < a.S; ++s) {
            B.scene = s;
            k_bptt<<<1, NTb, kBpttSmem, st>>>(B);
        }
    } else {
        k_bptt<<<grid, NTb, kBpttSmem, st>>>(B);
    }
    return cudaGetLastError();
}

cudaError_t launch_record(const StepArgs& a, float* ckpt, int ck, double* loss, int metrics, int16_t* rec_ov,
                          int32_t* rec_off, float lambda, float tau, int grid, cudaStream_t st) {
    BpttArgs B = bptt_args(a, ckpt, nullptr, ck, lambda, tau);
    B.loss = loss;
    B.metrics = metrics;
    B.rec_ov = rec_ov;
    B.rec_off = rec_off;
    cudaError_t e = cudaFuncSetAttribute(k_record, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kRecordSmem));
    if (e != cudaSuccess) return e;
    k_record<<<grid, NTb, kRecordSmem, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_backward(const StepArgs& a, float* ckpt, float* segbuf, int ck, const int16_t* rec_ov,
                            const int32_t* rec_off, const float* g_logdiv, const float* g_ov, const float* g_off,
                            const double* loss_w, float* dact, const StateP& dst0, float lambda, float tau, int grid,
                            cudaStream_t st) {
    BpttArgs B = bptt_args(a, ckpt, segbuf, ck, lambda, tau);
    B.rec_ov = const_cast<int16_t*>(rec_ov);
    B.rec_off = const_cast<int32_t*>(rec_off);
    B.g_logdiv = g_logdiv;
    B.g_ov = g_ov;
    B.g_off = g_off;
    B.loss_w = loss_w;
    B.dact = dact;
    B.dst0 = dst0;
    cudaError_t e = cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kBpttSmem));
    if (e != cudaSuccess) return e;
    k_backward<<<grid, NTb, kBpttSmem, st>>>(B);
    return cudaGetLastError();
}

// Resident CTAs per SM of the BPTT kernels (which = 0: k_bptt and
// k_backward; 1: k_record).
int bptt_blocks_per_sm(int which) {
    int n = 0;
    const void* f = which == 1 ? reinterpret_cast<const void*>(k_record) : reinterpret_cast<const void*>(k_bptt);
    const size_t smem = which == 1 ? kRecordSmem : kBpttSmem;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, NTb, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace wsim
