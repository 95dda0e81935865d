// Phases of one simulated step of one scene, shared by the per-step kernel,
// the plain per-scene kernels and the scene-resident rollout kernel.  A CTA
// of NT threads owns one scene; agent data lives in an AgentSmem block.
#pragma once
#include <math_constants.h>

#include "wsim_device.cuh"

namespace wsim {

#define WSIM_INF CUDART_INF_F
constexpr unsigned kFull = 0xffffffffu;

struct __align__(16) AgentSmem {
    uint64_t bar[2];
    unsigned long long cnt[kCounters];
    // current state (t during the transition, t+1 after the writeback)
    float xh[kMaxN], xl[kMaxN], yh[kMaxN], yl[kMaxN], c[kMaxN], s[kMaxN], hl[kMaxN], hw[kMaxN];
    float vx[kMaxN], vy[kMaxN], thh[kMaxN], thl[kMaxN], sh[kMaxN], sl[kMaxN];
    // next state
    float nxh[kMaxN], nxl[kMaxN], nyh[kMaxN], nyl[kMaxN], nth[kMaxN], ntl[kMaxN];
    float nvx[kMaxN], nvy[kMaxN], nsh[kMaxN], nsl[kMaxN];
    float off[kMaxN];
    uint32_t ovk[kMaxN];      // ov as an ordered key (max over the pair depths, atomicMax)
    uint32_t pk[kMaxN];       // the same with its low 8 bits replaced by the pair's other agent
    float4 obox[kMaxN];       // overlap culling record: (x, y, R, R - lower bound of ov)
    int32_t hint[4 * kMaxN];  // scene-resident nearest-segment cache
    int32_t ro[kMaxN + 1];    // the scene's route offsets (route_off of its agents and the end)
    float v0[kMaxN];          // IDM desired speeds
    uint8_t kind[kMaxN];
    uint8_t valid[kMaxN];
    uint8_t kin[kMaxN];       // kinematically infeasible transition into the current state
    int scene;
    int reward;
    int work[3];              // counters of the warp phases (transition, overlap rows, off-road groups)
};

// Work counters of one thread (flushed into the CTA's AgentSmem::cnt).
struct Counts {
    // 32 bits per thread: a thread's share of one launch stays far below 2^32
    uint32_t evals = 0, tiles = 0, pairs = 0, tests = 0, bounds = 0, filters = 0;
};

// One scene's packed road-edge segments, in global or shared memory.
struct SegView {
    const float4* geo;
    const float* inv;
    const uint8_t* flags;
    const float4* tiles;  // 2 per tile: capsule (start, chord), (radius, 1/|chord|^2)
    const float4* sup;    // bounding box per super-tile of kSuper tiles
    int E, nt, ns;
    const uint16_t* perm;  // the tiles in super-tile order (null: identity); lists stay in index order
};


// Order-preserving unsigned key of a float (atomicMax in shared memory).
// A pair depth and the pair's other agent share one key in pk: the depth's
// key with its low 8 bits replaced by the agent (the deepest partner to
// within 2^-16 relative, good enough to seed the next step's bound).
__device__ __forceinline__ uint32_t ukey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unukey(uint32_t k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }
__device__ __forceinline__ uint32_t partner_key(float d, int j) { return (ukey(d) & 0xffffff00u) | static_cast<uint32_t>(j); }
constexpr uint32_t kNoDepth = 0x007fffffu;  // ukey(-inf)

// Next agent of a warp phase (dynamic assignment balances uneven agents).
__device__ __forceinline__ int next_agent(AgentSmem& sm, int slot, int lane) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&sm.work[slot], 1);
    return __shfl_sync(0xffffffffu, i, 0);
}

// sqrt within a few float32 ulps (bounds and margins only; not for results).
__device__ __forceinline__ float sqrt_approx(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

template <class T> __device__ __forceinline__ T pick4(const T (&a)[4], int k) {
    return k == 0 ? a[0] : (k == 1 ? a[1] : (k == 2 ? a[2] : a[3]));
}

// ---------------------------------------------------------------------------
// Inverse kinematics of the bicycle action space (App. A.1) from two
// consecutive states: a = (|v'| - |v|) / dt (a product with 1/dt, within an
// ulp of the quotient); the direction of travel turns from the old heading
// to atan2(vy', vx') (the paper prints arctan(vx'/vy'): components swapped,
// quadrant lost), reduced modulo 2 pi; a state with zero velocity has no
// direction (turn 0); kappa = turn / (v dt + a dt^2 / 2), 0 when no
// distance is travelled.  dist is formed exactly as the forward model forms
// it, so an expert action turns the heading by `turn` to a few ulps.  The
// float32 atan2 and quotients are the fast forms (atan2_poly, 2-ulp
// division): the inverse is most of the open-loop expert kernel's issue.
// ---------------------------------------------------------------------------
constexpr float kTwoPiHi = 6.28318548202514648f;      // float nearest 2 pi
constexpr float kTwoPiLo = -1.74845553146951715e-7f;  // 2 pi - kTwoPiHi
constexpr float kInvTwoPi = 0.159154943091895336f;

// phi - (thh + thl) reduced modulo 2 pi (about [-pi, pi]); thh may be large.
__device__ __forceinline__ float turn_from(float phi, float thh, float thl) {
    float dh, dl;
    two_sum(phi, -thh, dh, dl);
    dl = __fsub_rn(dl, thl);
    const float k = rintf(dh * kInvTwoPi);
    const float r = fmaf(-k, kTwoPiHi, dh);  // one rounding of an almost exact difference
    return fmaf(-k, kTwoPiLo, r) + dl;
}

// atan2(y, x) in float32 for finite arguments: the octant reduction t =
// min(|x|, |y|) / max(|x|, |y|) in [0, 1], atan(t) = t P(t^2) with P of
// degree 7 (coefficients fitted by Lawson's iteratively reweighted least
// squares for the smallest largest relative error on [0, 1], 1e-7;
// gen_atan_poly.py beside this file), then atan(1/t) = pi/2 - atan(t),
// atan2(y, -x) = pi - atan2(y, x) and the sign of y.  Within 4e-7 rad of
// the exact angle (the quotient is an approximate division, 2 ulps);
// (0, 0) gives 0 and (+-0, x < 0) +-pi.
__device__ __forceinline__ float atan2_poly(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float s = t * t;
    float q = -4.693275783e-03f;
    q = fmaf(q, s, 2.425240166e-02f);
    q = fmaf(q, s, -5.948639289e-02f);
    q = fmaf(q, s, 9.914292395e-02f);
    q = fmaf(q, s, -1.401948035e-01f);
    q = fmaf(q, s, 1.996972412e-01f);
    q = fmaf(q, s, -3.333199024e-01f);
    q = fmaf(q, s, 9.999998808e-01f);
    float r = t * q;
    r = ay > ax ? 1.57079637f - r : r;   // float nearest pi/2
    r = x < 0.f ? 3.14159274f - r : r;   // float nearest pi
    return copysignf(r, y);
}

struct BicycleInv {
    float a, kappa, turn, dist;
};

// The same from the two speeds v = |(vx, vy)| and vn = |(nvx, nvy)| (callers
// that already hold them).
__device__ __forceinline__ BicycleInv bicycle_inverse_v(const Params& p, float v, float vn, float thh, float thl,
                                                        float nvx, float nvy) {
    BicycleInv r;
    r.a = (vn - v) * p.inv_dt;
    r.turn = (nvx != 0.f || nvy != 0.f) ? turn_from(atan2_poly(nvy, nvx), thh, thl) : 0.f;
    r.dist = fmaf(v, p.dt, r.a * (0.5f * p.dt * p.dt));
    r.kappa = r.dist > 0.f ? __fdividef(r.turn, r.dist) : 0.f;  // 2 ulps
    return r;
}

__device__ __forceinline__ BicycleInv bicycle_inverse(const Params& p, float vx, float vy, float thh, float thl,
                                                      float nvx, float nvy) {
    return bicycle_inverse_v(p, sqrtf(fmaf(vx, vx, vy * vy)), sqrtf(fmaf(nvx, nvx, nvy * nvy)), thh, thl, nvx, nvy);
}

// Discrete action grids (Sec. 5.2): n values over [-max, max], centred on 0
// for odd n.  Index rint(fl(v / step) + c) clamped to [0, n-1]; value
// fl((i - c) * step); step = fl(2 max / (n-1)), c = (n-1)/2.
__device__ __forceinline__ int disc_index(float v, float max, int n) {
    const float step = __fdiv_rn(2.0f * max, static_cast<float>(n - 1));
    const float c = 0.5f * static_cast<float>(n - 1);
    const float q = __fadd_rn(__fdiv_rn(v, step), c);
    return static_cast<int>(fminf(static_cast<float>(n - 1), fmaxf(0.f, rintf(q))));
}
__device__ __forceinline__ float disc_value(int i, float max, int n) {
    const float step = __fdiv_rn(2.0f * max, static_cast<float>(n - 1));
    const float c = 0.5f * static_cast<float>(n - 1);
    return __fmul_rn(__fsub_rn(static_cast<float>(i), c), step);
}
// Flat index of an action (u0, u1, u2) of agent kind `kind` (-1 for IDM).
__device__ __forceinline__ int disc_encode(const Params& p, int kind, float u0, float u1, float u2) {
    if (kind == WSIM_KIND_BICYCLE) return disc_index(u0, p.da_max, p.na) * p.nk + disc_index(u1, p.dk_max, p.nk);
    if (kind == WSIM_KIND_DELTA)
        return (disc_index(u0, p.dd_max, p.nd) * p.nd + disc_index(u1, p.dd_max, p.nd)) * p.nt +
               disc_index(u2, p.dt_max, p.nt);
    return -1;
}
// The grid action of flat index idx (false when idx lies past the grid).
__device__ __forceinline__ bool disc_decode(const Params& p, int kind, int idx, float& u0, float& u1, float& u2) {
    u0 = u1 = u2 = 0.f;
    if (idx < 0) return true;
    if (kind == WSIM_KIND_BICYCLE) {
        if (idx >= p.na * p.nk) return false;
        u0 = disc_value(idx / p.nk, p.da_max, p.na);
        u1 = disc_value(idx % p.nk, p.dk_max, p.nk);
    } else if (kind == WSIM_KIND_DELTA) {
        if (idx >= p.nd * p.nd * p.nt) return false;
        const int it = idx % p.nt, ixy = idx / p.nt;
        u0 = disc_value(ixy / p.nd, p.dd_max, p.nd);
        u1 = disc_value(ixy % p.nd, p.dd_max, p.nd);
        u2 = disc_value(it, p.dt_max, p.nt);
    }
    return true;
}

// Sec. 3.4 kinematic infeasibility of a transition: the inverse kinematics
// break |a| <= kin_amax or |kappa| <= kin_kmax (the curvature test with the
// distance multiplied out, defined for any step length).
__device__ __forceinline__ uint8_t kin_infeasible(const Params& p, float vx, float vy, float thh, float thl,
                                                  float nvx, float nvy) {
    const BicycleInv r = bicycle_inverse(p, vx, vy, thh, thl, nvx, nvy);
    return fabsf(r.a) > p.kin_amax || fabsf(r.turn) > p.kin_kmax * r.dist;
}

// ---------------------------------------------------------------------------
// Loading and storing agent state.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void load_state(AgentSmem& sm, const StepArgs& A, const CStateP& st, int a0, int N) {
    for (int i = threadIdx.x; i < N; i += NT) {
        const int g = a0 + i;
        sm.xh[i] = st.x[g];
        sm.xl[i] = st.x_lo[g];
        sm.yh[i] = st.y[g];
        sm.yl[i] = st.y_lo[g];
        const float th = st.th[g], tl = st.th_lo[g];
        sm.thh[i] = th;
        sm.thl[i] = tl;
        float c, s;
        comp_sincos(th, tl, c, s);
        sm.c[i] = c;
        sm.s[i] = s;
        sm.hl[i] = 0.5f * A.L[g];
        sm.hw[i] = 0.5f * A.W[g];
        sm.vx[i] = st.vx[g];
        sm.vy[i] = st.vy[g];
        sm.sh[i] = st.s[g];
        sm.sl[i] = st.s_lo[g];
        sm.valid[i] = A.valid[g];
        // per-agent constants the transitions read every step (absent in a
        // metrics-only batch)
        sm.kind[i] = A.kind ? A.kind[g] : static_cast<uint8_t>(WSIM_KIND_BICYCLE);
        sm.v0[i] = A.v0 ? A.v0[g] : 0.f;
        sm.ro[i] = A.route_off ? A.route_off[g] : 0;
        sm.kin[i] = 0;
        sm.ovk[i] = kNoDepth;
        sm.pk[i] = kNoDepth;
        // culling record of the loaded state (no lower bound yet); the IDM
        // candidate filter reads its centre and R >= hl + hw
        const float R = (sm.hl[i] + sm.hw[i]) * 1.000001f + 5e-4f;
        sm.obox[i] = sm.valid[i] ? make_float4(st.x[g], st.y[g], R, -WSIM_INF)
                                 : make_float4(st.x[g], st.y[g], -WSIM_INF, -WSIM_INF);
    }
    if (threadIdx.x == 0) {
        sm.work[0] = sm.work[1] = sm.work[2] = 0;
        sm.ro[N] = A.route_off ? A.route_off[a0 + N] : 0;
    }
}

// Make the next state current (after flagging a kinematically infeasible
// transition); optionally store it to global memory.  Runs between barriers
// after the transition, so it also rearms the transition's agent counter for
// the next step.
template <int NT>
__device__ void writeback(AgentSmem& sm, const Params& p, const StateP* out, int a0, int N) {
    if (threadIdx.x == 0) sm.work[0] = 0;
    for (int i = threadIdx.x; i < N; i += NT) {
        sm.kin[i] = sm.valid[i] ? kin_infeasible(p, sm.vx[i], sm.vy[i], sm.thh[i], sm.thl[i], sm.nvx[i], sm.nvy[i])
                                : uint8_t(0);
        if (out) {
            const int g = a0 + i;
            out->x[g] = sm.nxh[i];
            out->x_lo[g] = sm.nxl[i];
            out->y[g] = sm.nyh[i];
            out->y_lo[g] = sm.nyl[i];
            out->th[g] = sm.nth[i];
            out->th_lo[g] = sm.ntl[i];
            out->vx[g] = sm.nvx[i];
            out->vy[g] = sm.nvy[i];
            out->s[g] = sm.nsh[i];
            out->s_lo[g] = sm.nsl[i];
        }
        sm.xh[i] = sm.nxh[i];
        sm.xl[i] = sm.nxl[i];
        sm.yh[i] = sm.nyh[i];
        sm.yl[i] = sm.nyl[i];
        sm.thh[i] = sm.nth[i];
        sm.thl[i] = sm.ntl[i];
        float c, s;
        comp_sincos(sm.nth[i], sm.ntl[i], c, s);
        sm.c[i] = c;
        sm.s[i] = s;
        sm.vx[i] = sm.nvx[i];
        sm.vy[i] = sm.nvy[i];
        sm.sh[i] = sm.nsh[i];
        sm.sl[i] = sm.nsl[i];
        sm.obox[i].x = sm.nxh[i];  // the culling record's centre follows the state
        sm.obox[i].y = sm.nyh[i];
    }
}

// Store the current state to global memory.
template <int NT>
__device__ void store_state(const AgentSmem& sm, const StateP& out, int a0, int N) {
    for (int i = threadIdx.x; i < N; i += NT) {
        const int g = a0 + i;
        out.x[g] = sm.xh[i];
        out.x_lo[g] = sm.xl[i];
        out.y[g] = sm.yh[i];
        out.y_lo[g] = sm.yl[i];
        out.th[g] = sm.thh[i];
        out.th_lo[g] = sm.thl[i];
        out.vx[g] = sm.vx[i];
        out.vy[g] = sm.vy[i];
        out.s[g] = sm.sh[i];
        out.s_lo[g] = sm.sl[i];
    }
}

// ---------------------------------------------------------------------------
// Route polyline: parameter (hi + lo) -> segment index and fraction.
// Segment k = floor(s / h), clamped to the route; beyond either end the
// fraction leaves [0, 1) so the end segment is extrapolated.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void route_locate(float hi, float lo, const Params& p, int P, int& seg, float& tau) {
    const float u = hi * p.inv_h;
    const float fl = floorf(u);
    tau = fmaf(lo, p.inv_h, u - fl);
    seg = static_cast<int>(fl);
    if (tau < 0.f) {
        seg -= 1;
        tau += 1.f;
    } else if (tau >= 1.f) {
        seg += 1;
        tau -= 1.f;
    }
    if (seg < 0) {
        tau += static_cast<float>(seg);
        seg = 0;
    }
    if (seg > P - 2) {
        tau += static_cast<float>(seg - (P - 2));
        seg = P - 2;
    }
}

// ---------------------------------------------------------------------------
// IDM route following (Sec. 3.5; textbook IDM of Treiber et al.) of the
// agents i0 .. i0+kIdmGroup-1 that follow their route, one warp per group.
// The per-agent arithmetic (route cursor, acceleration, advance) runs one
// lane per agent; the lead search runs warp-wide, agent by agent: lane k
// holds look-ahead sample k+1 at route parameter s + L/2 + dq (k+1).
// Candidate agents are found 32 at a time (one per lane) by a bounding-circle
// test; for each candidate the warp tests all 32 samples against its box
// widened by half this agent's width, and the ballot's lowest set bit is the
// first hit.  The lead is the hit agent with the smallest bumper gap (ties:
// lower index).
// ---------------------------------------------------------------------------
constexpr int kIdmGroup = 8;

__device__ __forceinline__ int ctrl_of(const StepArgs& A, int g) {
    return A.ctrl ? A.ctrl[g] : WSIM_CTRL_ACTION;
}

// Whether agent i is advanced by IDM in this transition.
__device__ __forceinline__ bool idm_moves(const AgentSmem& sm, const StepArgs& A, int a0, int i) {
    return sm.kind[i] == WSIM_KIND_IDM && sm.valid[i] && ctrl_of(A, a0 + i) != WSIM_CTRL_LOG;
}

struct IdmLead {
    int lead;         // -1: no lead
    float gap;        // bumper gap to the lead
    float tlx, tly;   // route tangent at the first sample inside the lead's box
};

// Look-ahead sample k (0-based; at route parameter s + L/2 + dq (k+1)) of an
// IDM agent with route cursor (sh, sl) and half length hl: the route point
// (Px, Py) starting its segment, the segment vector (dx, dy) and the offset
// (qox, qoy) = tau (dx, dy) of the sample along it.
struct IdmSample {
    float Px, Py, dx, dy, qox, qoy;
};
__device__ __forceinline__ IdmSample idm_sample(const Params& p, const float* rx, const float* ry, int P, float sh,
                                                float sl, float hl, int k) {
    float bh, bl;
    two_sum(sh, fmaf(p.dq, static_cast<float>(k + 1), hl), bh, bl);
    bl = __fadd_rn(bl, sl);
    int seg;
    float tau;
    route_locate(bh, bl, p, P, seg, tau);
    IdmSample q;
    q.Px = rx[seg];
    q.Py = ry[seg];
    q.dx = rx[seg + 1] - q.Px;
    q.dy = ry[seg + 1] - q.Py;
    q.qox = tau * q.dx;
    q.qoy = tau * q.dy;
    return q;
}

// Whether look-ahead sample (P + qo) lies in agent j's box widened by wi
// (half the follower's width) on both axes.
__device__ __forceinline__ bool idm_in_box(const AgentSmem& sm, int j, float Px, float Py, float qox, float qoy,
                                           float wi) {
    const float rxq = (Px - sm.xh[j]) + (qox - sm.xl[j]);
    const float ryq = (Py - sm.yh[j]) + (qoy - sm.yl[j]);
    const float cj = sm.c[j], sj = sm.s[j];
    const float pu = fabsf(fmaf(rxq, cj, ryq * sj));
    const float pn = fabsf(fmaf(-rxq, sj, ryq * cj));
    return fminf(sm.hl[j] + wi - pu, sm.hw[j] + wi - pn) >= 0.f;
}

// Bumper gap between follower i and agent j (clamped below at gap_min).
__device__ __forceinline__ float idm_gap(const AgentSmem& sm, const Params& p, int i, int j) {
    const float ddx = comp_diff(sm.xh[j], sm.xl[j], sm.xh[i], sm.xl[i]);
    const float ddy = comp_diff(sm.yh[j], sm.yl[j], sm.yh[i], sm.yl[i]);
    return fmaxf(p.gap_min, sqrtf(fmaf(ddx, ddx, ddy * ddy)) - (sm.hl[i] + sm.hl[j]));
}

// Lead of agent i (warp-wide; every lane returns the same result).
static __device__ IdmLead idm_lead(AgentSmem& sm, const StepArgs& A, int a0, int N, int i, int lane, Counts& cnt) {
    const Params& p = A.p;
    const int ro = sm.ro[i];
    const int P = sm.ro[i + 1] - ro;
    const float* rx = A.route_x + ro;
    const float* ry = A.route_y + ro;
    const float hli = sm.hl[i], wi = sm.hw[i];

    // This lane's look-ahead sample.
    const IdmSample smp = idm_sample(p, rx, ry, P, sm.sh[i], sm.sl[i], hli, lane);
    const float Px = smp.Px, Py = smp.Py, dx = smp.dx, dy = smp.dy, qox = smp.qox, qoy = smp.qoy;

    // Bounding circles of the four groups of 8 consecutive samples, centred
    // on each group's fifth sample: the samples of a group lie within 4 dq
    // of route parameter of it, so within 4 dq rf in the plane (rf: the
    // route's largest segment length per route parameter); a box (widened
    // by wi) that holds a sample of group G has its centre within that
    // radius + hl + hw + 2 wi of the circle's centre (5 cm of slack for the
    // float32 positions).
    const float qx = Px + qox, qy = Py + qoy;
    // (read from global memory beside the route loads: a per-agent array in
    // shared memory would cost a four-CTA shape its shared-memory carve-out)
    const float rf = A.route_rf ? A.route_rf[a0 + i] : WSIM_INF;
    const float gr = fmaf(4.f * p.dq, rf, 2.f * wi + 0.05f);
    float cxs[4], cys[4], crs[4];  // the four circles in every lane
#pragma unroll
    for (int G = 0; G < 4; ++G) {
        cxs[G] = __shfl_sync(kFull, qx, 8 * G + 4);
        cys[G] = __shfl_sync(kFull, qy, 8 * G + 4);
        crs[G] = gr;
    }

    int lead = -1, lead_hit = 0;
    float gbest = WSIM_INF;
    // Samples in the widened box of agent j (one ballot bit per sample).
    auto box_hits = [&](int j) { return idm_in_box(sm, j, Px, Py, qox, qoy, wi); };
    auto take = [&](int j, unsigned hits) {
        const float gap = idm_gap(sm, p, i, j);
        if (gap < gbest) {
            gbest = gap;
            lead = j;
            lead_hit = __ffs(hits) - 1;
        }
    };
    for (int jb = 0; jb < N; jb += 32) {
        const int jl = jb + lane;
        bool cand = false;
        // non-candidates test a point that no circle reaches; the culling
        // record gives the centre and R >= hl + hw in one load (a wider
        // reach only adds candidates that the box tests reject)
        float xj = WSIM_INF, yj = WSIM_INF, reach = 0.f;
        if (jl < N && jl != i) {
            const float4 P = sm.obox[jl];
            if (P.z > 0.f) {  // valid
                xj = P.x;
                yj = P.y;
                reach = P.z;
            }
        }
        cnt.filters += 4;
#pragma unroll
        for (int G = 0; G < 4; ++G) {
            const float ex = xj - cxs[G], ey = yj - cys[G];
            const float rr = crs[G] + reach;
            cand = cand || fmaf(ex, ex, ey * ey) <= rr * rr;
        }
        unsigned cm = __ballot_sync(kFull, cand);
        // Two candidates per iteration (independent tests), taken in index
        // order so that ties go to the lower index.
        while (cm) {
            const int j1 = jb + __ffs(cm) - 1;
            cm &= cm - 1;
            const bool two = cm != 0;
            const int j2 = two ? jb + __ffs(cm) - 1 : j1;
            if (two) cm &= cm - 1;
            if (lane == 0) cnt.tests += two ? 64 : 32;
            const bool in1 = box_hits(j1), in2 = box_hits(j2);
            const unsigned h1 = __ballot_sync(kFull, in1);
            const unsigned h2 = __ballot_sync(kFull, in2 && two);
            if (h1) take(j1, h1);
            if (h2) take(j2, h2);
        }
    }
    const float rn = rsqrtf(fmaf(dx, dx, dy * dy));
    const float tlx = __shfl_sync(kFull, dx * rn, lead_hit), tly = __shfl_sync(kFull, dy * rn, lead_hit);
    return IdmLead{lead, gbest, tlx, tly};
}

// IDM acceleration (exponent 4) of agent i with lead L (the lead's velocity
// (lvx, lvy) at t), then the advance along its route into the n* arrays.
static __device__ void idm_accel_advance(AgentSmem& sm, const StepArgs& A, int a0, int i, const IdmLead& L, float lvx,
                                         float lvy) {
    const Params& p = A.p;
    const float vxi = sm.vx[i], vyi = sm.vy[i];
    const float v = sqrtf(fmaf(vxi, vxi, vyi * vyi));
    const float r = v / sm.v0[i];
    const float r2 = r * r;
    const float r4 = r2 * r2;
    float acc;
    if (L.lead >= 0) {
        const float vl = fmaf(lvx, L.tlx, lvy * L.tly);
        const float sstar = p.s0 + fmaxf(0.f, fmaf(v, p.T, v * (v - vl) / p.idm_sqrt_ab2));
        const float q = sstar / L.gap;
        acc = p.amax * (1.f - r4 - q * q);
    } else {
        acc = p.amax * (1.f - r4);
    }
    // Advance along the route by the trapezoidal distance of the new speed.
    const int ro = sm.ro[i];
    const int P = sm.ro[i + 1] - ro;
    const float vn = fmaxf(0.f, fmaf(acc, p.dt, v));
    float sh = sm.sh[i], sl = sm.sl[i];
    comp_add(sh, sl, 0.5f * (v + vn) * p.dt);
    int sg;
    float ta;
    route_locate(sh, sl, p, P, sg, ta);
    const float Qx = A.route_x[ro + sg], Qy = A.route_y[ro + sg];
    const float ux = A.route_x[ro + sg + 1] - Qx, uy = A.route_y[ro + sg + 1] - Qy;
    float xh, xe, yh, ye;
    two_sum(Qx, ta * ux, xh, xe);
    two_sum(Qy, ta * uy, yh, ye);
    const float un = rsqrtf(fmaf(ux, ux, uy * uy));
    sm.nxh[i] = xh;
    sm.nxl[i] = xe;
    sm.nyh[i] = yh;
    sm.nyl[i] = ye;
    sm.nth[i] = atan2f(uy, ux);
    sm.ntl[i] = 0.f;
    sm.nvx[i] = vn * ux * un;
    sm.nvy[i] = vn * uy * un;
    sm.nsh[i] = sh;
    sm.nsl[i] = sl;
}

static __device__ void idm_group(AgentSmem& sm, const StepArgs& A, int a0, int N, int i0, int lane, Counts& cnt) {
    const int i = i0 + lane;
    const bool mine = lane < kIdmGroup && i < N && idm_moves(sm, A, a0, i);
    IdmLead L{-1, WSIM_INF, 0.f, 0.f};
    for (unsigned todo = __ballot_sync(kFull, mine); todo; todo &= todo - 1) {
        const int k = __ffs(todo) - 1;
        const IdmLead l = idm_lead(sm, A, a0, N, i0 + k, lane, cnt);
        if (lane == k) L = l;
    }
    if (!mine) return;
    idm_accel_advance(sm, A, a0, i, L, L.lead >= 0 ? sm.vx[L.lead] : 0.f, L.lead >= 0 ? sm.vy[L.lead] : 0.f);
}

// ---------------------------------------------------------------------------
// Transition t -> t+1 of one scene into the n* arrays.  act is [3][N_tot]
// (null when no agent takes WSIM_CTRL_ACTION); t_next = t+1 is the log row
// read by the expert and by log playback.
// ---------------------------------------------------------------------------

// IDM agents of the transition, kIdmGroup agents per warp task, taken from work[0].
__device__ __forceinline__ void transition_idm_tasks(AgentSmem& sm, const StepArgs& A, int a0, int N, Counts& cnt) {
    const int lane = threadIdx.x & 31;
    for (int q = next_agent(sm, 0, lane); q * kIdmGroup < N; q = next_agent(sm, 0, lane))
        idm_group(sm, A, a0, N, q * kIdmGroup, lane, cnt);
}

template <int NT, bool DRIVERS = true>
__device__ void transition_policy(AgentSmem& sm, const StepArgs& A, const float* act, int t_next, int a0, int N);

template <int NT>
__device__ void phase_transition(AgentSmem& sm, const StepArgs& A, const float* act, int t_next, int a0, int N,
                                 Counts& cnt) {
    if (threadIdx.x == 0) sm.work[1] = sm.work[2] = 0;  // the metrics phase starts after two barriers
    transition_idm_tasks(sm, A, a0, N, cnt);
    transition_policy<NT>(sm, A, act, t_next, a0, N);
}

// Every agent that is not an IDM agent on its route, one thread each: the
// policy dynamics (given action, expert, discrete expert), log playback, or
// a copy of the state.  DRIVERS = false compiles the given-action driver
// only (A.ctrl must be null), which keeps the rollout kernel's code small.
template <int NT, bool DRIVERS>
__device__ void transition_policy(AgentSmem& sm, const StepArgs& A, const float* act, int t_next, int a0, int N) {
    const Params& p = A.p;
    const bool full_log = A.log_th && A.log_vx && A.log_vy;
    const size_t row = static_cast<size_t>(t_next) * A.N_tot;
    for (int i = threadIdx.x; i < N; i += NT) {
        const int g = a0 + i;
        const int kind = sm.kind[i];
        const int cm = DRIVERS ? ctrl_of(A, g) : WSIM_CTRL_ACTION;
        if (kind == WSIM_KIND_IDM && sm.valid[i] && cm != WSIM_CTRL_LOG) continue;
        float xh = sm.xh[i], xl = sm.xl[i], yh = sm.yh[i], yl = sm.yl[i];
        float thh = sm.thh[i], thl = sm.thl[i];
        float vx = sm.vx[i], vy = sm.vy[i];
        const bool expert = cm == WSIM_CTRL_EXPERT || cm == WSIM_CTRL_EXPERT_DISCRETE;
        bool moves = sm.valid[i] && (cm == WSIM_CTRL_LOG || (kind != WSIM_KIND_IDM && cm != WSIM_CTRL_HOLD));
        if (moves && (cm > WSIM_CTRL_EXPERT_DISCRETE || (cm == WSIM_CTRL_ACTION && !act) ||
                      ((expert || cm == WSIM_CTRL_LOG) && !full_log))) {
            set_status(A.status, WSIM_EINVAL);
            moves = false;
        }
        if (moves && cm == WSIM_CTRL_LOG) {
            // Log playback (Sec. 3.5): the logged state of t+1.
            xh = A.log_x[row + g];
            yh = A.log_y[row + g];
            thh = A.log_th[row + g];
            xl = yl = thl = 0.f;
            vx = A.log_vx[row + g];
            vy = A.log_vy[row + g];
        } else if (moves && kind == WSIM_KIND_BICYCLE) {
            // App. A.1 bicycle forward dynamics; the expert (Sec. 5.2) first
            // fits (a, kappa) to the logged velocity of t+1.
            float a, k;
            if (expert) {
                const BicycleInv r = bicycle_inverse(p, vx, vy, thh, thl, A.log_vx[row + g], A.log_vy[row + g]);
                a = r.a;
                k = r.kappa;
                if (cm == WSIM_CTRL_EXPERT_DISCRETE) {  // snapped to the discrete grid
                    float unused;
                    disc_decode(p, kind, disc_encode(p, kind, a, k, 0.f), a, k, unused);
                }
            } else {
                a = act[g];
                k = act[A.N_tot + g];
            }
            if (!isfinite(a) || !isfinite(k)) set_status(A.status, WSIM_ENONFINITE);
            const float v = sqrtf(fmaf(vx, vx, vy * vy));
            const float ah = a * (0.5f * p.dt * p.dt);
            comp_add(xh, xl, fmaf(vx, p.dt, ah * sm.c[i]));
            comp_add(yh, yl, fmaf(vy, p.dt, ah * sm.s[i]));
            comp_add(thh, thl, k * fmaf(v, p.dt, ah));
            const float vn = fmaf(a, p.dt, v);
            float cn, sn;
            comp_sincos(thh, thl, cn, sn);
            vx = vn * cn;
            vy = vn * sn;
        } else if (moves && kind == WSIM_KIND_DELTA) {
            // App. A.1 delta dynamics; the expert's displacement (Sec. 5.2)
            // is the delta inverse, log row t+1 minus the state.
            float ddx, ddy, dth;
            if (expert) {
                ddx = __fsub_rn(A.log_x[row + g] - xh, xl);
                ddy = __fsub_rn(A.log_y[row + g] - yh, yl);
                dth = __fsub_rn(A.log_th[row + g] - thh, thl);
                if (cm == WSIM_CTRL_EXPERT_DISCRETE)  // snapped to the discrete grid
                    disc_decode(p, kind, disc_encode(p, kind, ddx, ddy, dth), ddx, ddy, dth);
            } else {
                ddx = act[g];
                ddy = act[A.N_tot + g];
                dth = act[2 * A.N_tot + g];
            }
            if (!isfinite(ddx) || !isfinite(ddy) || !isfinite(dth)) set_status(A.status, WSIM_ENONFINITE);
            comp_add(xh, xl, ddx);
            comp_add(yh, yl, ddy);
            comp_add(thh, thl, dth);
            vx = ddx / p.dt;
            vy = ddy / p.dt;
        }
        sm.nxh[i] = xh;
        sm.nxl[i] = xl;
        sm.nyh[i] = yh;
        sm.nyl[i] = yl;
        sm.nth[i] = thh;
        sm.ntl[i] = thl;
        sm.nvx[i] = vx;
        sm.nvy[i] = vy;
        sm.nsh[i] = sm.sh[i];
        sm.nsl[i] = sm.sl[i];
    }
}

// ---------------------------------------------------------------------------
// Overlap, row i (warp): the SAT depth d_ij of every valid j > i, computed once
// per unordered pair with i as the first box (the canonical order, so that
// d_ij is one value for both agents), folded into both agents' maxima (ovk)
// and partner keys (pk) by atomicMax.  ov_i = max over all valid j != i.
//
// Culling (exact): d_ij <= R_i + R_j - |c_j - c_i| / sqrt(2), where R = half
// length + half width bounds the half diagonal (one of box i's two axes takes
// at least |dc| / sqrt(2) of the centre distance).  lb_i <= ov_i is the depth
// against last step's deepest partner, so a pair whose bound lies below both
// lb_i and lb_j changes neither maximum and is skipped (1.5 mm of slack for
// the float32 bound and the hi words used).
// ---------------------------------------------------------------------------
// Exact argmax key of a pair depth for agent records: the depth's ordered
// key above the partner's index complement, so that the maximum key names
// the deepest partner, ties to the lower index.  0 = no partner.
__device__ __forceinline__ unsigned long long argmax_key(float d, int j) {
    return (static_cast<unsigned long long>(ukey(d)) << 32) | static_cast<unsigned long long>(0xffffu - j);
}
__device__ __forceinline__ int argmax_partner(unsigned long long k) {
    return k ? static_cast<int>(0xffffu - static_cast<unsigned>(k & 0xffffu)) : -1;
}

// REC: also folds argmax_key into k64[] of both agents (records of the
// differentiable rollout; a culled pair cannot be a maximum, so the recorded
// partner is the exhaustive argmax).
template <bool REC = false>
static __device__ void overlap_row(AgentSmem& sm, int N, int i, int lane, Counts& cnt,
                                   unsigned long long* k64 = nullptr) {
    const float4 Pi = sm.obox[i];
    const float xih = sm.xh[i], xil = sm.xl[i], yih = sm.yh[i], yil = sm.yl[i];
    const float ci = sm.c[i], si = sm.s[i], hli = sm.hl[i], hwi = sm.hw[i];
    for (int j = i + 1 + lane; j < N; j += 32) {
        const float4 Pj = sm.obox[j];  // invalid agents: R = -inf, always skipped
        cnt.bounds += 1;
        const float dx = Pj.x - Pi.x, dy = Pj.y - Pi.y;
        const float t = fmaxf(Pi.w + Pj.z, Pi.z + Pj.w);  // |dc| / sqrt(2) above this: skip
        if (!(t >= 0.f) || fmaf(dx, dx, dy * dy) > 2.f * t * t) continue;
        const float ddx = comp_diff(sm.xh[j], sm.xl[j], xih, xil);
        const float ddy = comp_diff(sm.yh[j], sm.yl[j], yih, yil);
        const float d = sat_depth(ddx, ddy, ci, si, hli, hwi, sm.c[j], sm.s[j], sm.hl[j], sm.hw[j]);
        // both agents' maxima and partner keys (max is order-free)
        atomicMax(&sm.ovk[j], ukey(d));
        atomicMax(&sm.pk[j], partner_key(d, i));
        atomicMax(&sm.ovk[i], ukey(d));
        atomicMax(&sm.pk[i], partner_key(d, j));
        if (REC) {
            atomicMax(&k64[j], argmax_key(d, i));
            atomicMax(&k64[i], argmax_key(d, j));
        }
        cnt.pairs += 2;
    }
}

// The culling records (thread per agent, before the rows): lb_i is the depth
// of agent i against the partner its key names (the pair's canonical
// evaluation), -inf without one; then the maxima are reset for this step.
template <int NT>
__device__ void overlap_bounds(AgentSmem& sm, int N) {
    for (int i = threadIdx.x; i < N; i += NT) {
        float lb = -WSIM_INF;
        const int p = (sm.pk[i] >> 8) > (kNoDepth >> 8) ? static_cast<int>(sm.pk[i] & 0xffu) : -1;
        if (sm.valid[i] && p >= 0 && p < N && p != i && sm.valid[p]) {
            const int a = min(i, p), b = max(i, p);
            const float dx = comp_diff(sm.xh[b], sm.xl[b], sm.xh[a], sm.xl[a]);
            const float dy = comp_diff(sm.yh[b], sm.yl[b], sm.yh[a], sm.yl[a]);
            lb = sat_depth(dx, dy, sm.c[a], sm.s[a], sm.hl[a], sm.hw[a], sm.c[b], sm.s[b], sm.hl[b], sm.hw[b]);
        }
        const float R = (sm.hl[i] + sm.hw[i]) * 1.000001f + 5e-4f;
        sm.obox[i] = sm.valid[i] ? make_float4(sm.xh[i], sm.yh[i], R, R - lb + 5e-4f)
                                 : make_float4(sm.xh[i], sm.yh[i], -WSIM_INF, -WSIM_INF);
        sm.ovk[i] = kNoDepth;
        sm.pk[i] = kNoDepth;
    }
}

// Squared distance of point p to the chord of capsule record C (1/|chord|^2 = inv).
__device__ __forceinline__ float cap_d2(float4 C, float inv, float px, float py) {
    const float wx = px - C.x, wy = py - C.y;
    const float t = __saturatef(fmaf(wx, C.z, wy * C.w) * inv);
    const float ex = fmaf(-t, C.z, wx), ey = fmaf(-t, C.w, wy);
    return fmaf(ex, ex, ey * ey);
}

// Squared distance from corner (ch + cl) to segment G; raw projection in *traw.
__device__ __forceinline__ float seg_dist2(float4 G, float iv, float cxh, float cxl, float cyh, float cyl,
                                           float* traw = nullptr) {
    const float wx = (cxh - G.x) + cxl;
    const float wy = (cyh - G.y) + cyl;
    const float dot = fmaf(wx, G.z, wy * G.w) * iv;
    if (traw) *traw = dot;
    const float t = __saturatef(dot);
    const float ex = fmaf(-t, G.z, wx), ey = fmaf(-t, G.w, wy);
    return fmaf(ex, ex, ey * ey);
}

// Scan two tiles at once (lanes 0-15: tile ta, lanes 16-31: tile tb) for the
// corners in their masks, updating each lane's (distance, index) minima.
// TIE: the tiles may come in any order, so equal distances compare indexes
// (otherwise they come in increasing index order and the first one stays).
template <bool TIE = false>
__device__ __forceinline__ void scan_pair(const SegView& V, int lane, int ta, unsigned ma, int tb, unsigned mb,
                                          float xh, float yh, const float (&cxl)[4], const float (&cyl)[4],
                                          float (&bd)[4], int (&bi)[4], Counts& cnt) {
    const bool upper = lane >= kTile;
    const int t = upper ? tb : ta;
    const unsigned m = upper ? mb : ma;
    const unsigned u = ma | mb;
    const int e = t * kTile + (lane & (kTile - 1));
    if (lane == 0) cnt.evals += kTile * (__popc(ma) + __popc(mb));
    if (m) {  // positions up to the tile's end hold segments or far-away padding
        const float4 G = V.geo[e];
        const float iv = V.inv[e];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((u >> k) & 1u) {
                const float d2 = seg_dist2(G, iv, xh, cxl[k], yh, cyl[k]);
                if (((m >> k) & 1u) && (d2 < bd[k] || (TIE && d2 == bd[k] && e < bi[k]))) {
                    bd[k] = d2;
                    bi[k] = e;
                }
            }
        }
    }
}

// Takes up to two tiles from the ballot `want` (lane l's tile and corner mask
// in t_l, cm_l) and scans them.
template <bool TIE = false>
__device__ __forceinline__ void scan_next_two(const SegView& V, int lane, unsigned& want, int tl_lane,
                                              unsigned cm_lane, float xh, float yh, const float (&cxl)[4],
                                              const float (&cyl)[4], float (&bd)[4], int (&bi)[4], Counts& cnt) {
    const int l1 = __ffs(want) - 1;
    want &= want - 1;
    const int l2 = want ? __ffs(want) - 1 : l1;
    const bool two = want != 0;
    want &= want - 1;
    const unsigned m1 = __shfl_sync(kFull, cm_lane, l1);
    const int t1 = __shfl_sync(kFull, tl_lane, l1);
    const unsigned m2 = __shfl_sync(kFull, cm_lane, l2);
    const int t2 = __shfl_sync(kFull, tl_lane, l2);
    scan_pair<TIE>(V, lane, t1, m1, t2, two ? m2 : 0u, xh, yh, cxl, cyl, bd, bi, cnt);
}

// Ascending sort of one value per lane (bitonic network over the warp).
__device__ __forceinline__ unsigned warp_sort_asc(unsigned v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned o = __shfl_xor_sync(kFull, v, j);
            const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
            v = take_min ? min(v, o) : max(v, o);
        }
    return v;
}


// ---------------------------------------------------------------------------
// Off-road of agent i (warp; Sec. 3.4: the road lies left of an oriented road
// edge).  For each box corner: the nearest road-edge segment (exact, ties to
// the lower index) and the side of its nearest feature, with the vertex rule
// where that feature is a vertex shared by two segments.  Returns
// max over corners of the signed distance (+ = off road) in every lane.
//
// Culling: an upper bound U_k on corner k's nearest distance comes from the
// segment that was nearest at the previous step (hint) or, without one, from
// points known to lie on segments (two per tile).  Super-tiles (kSuper tiles)
// and then tiles whose bounding box lies farther than U_k from corner k are
// skipped; the rest are scanned with one segment per lane, so the result
// equals the exhaustive scan.  hint (may be null) is read and updated.
// ---------------------------------------------------------------------------
// Signed distance of a corner (xh + cl, yh + dl) whose nearest segment is e
// at squared distance d2: side of the nearest feature, with the vertex rule
// where that feature is a vertex shared by two segments.
__device__ __forceinline__ float corner_side(const SegView& V, int e, float d2, float xh, float cl, float yh,
                                             float dl) {
    const float4 G = V.geo[e];
    const uint8_t fl = V.flags[e];
    float traw;
    seg_dist2(G, V.inv[e], xh, cl, yh, dl, &traw);
    const float wx = (xh - G.x) + cl, wy = (yh - G.y) + dl;
    bool on;
    if (traw <= 0.f && (fl & 1)) {
        const float4 Gp = V.geo[e - 1];
        const bool l1 = fmaf(Gp.z, wy, -Gp.w * wx) > 0.f;
        const bool l2 = fmaf(G.z, wy, -G.w * wx) > 0.f;
        const float turn = fmaf(Gp.z, G.w, -Gp.w * G.z);
        on = turn > 0.f ? (l1 && l2) : (turn < 0.f ? (l1 || l2) : l1);
    } else if (traw >= 1.f && (fl & 2)) {
        const float4 Gn = V.geo[e + 1];
        const float qx = wx - G.z, qy = wy - G.w;
        const bool l1 = fmaf(G.z, qy, -G.w * qx) > 0.f;
        const bool l2 = fmaf(Gn.z, qy, -Gn.w * qx) > 0.f;
        const float turn = fmaf(G.z, Gn.w, -G.w * Gn.z);
        on = turn > 0.f ? (l1 && l2) : (turn < 0.f ? (l1 || l2) : l1);
    } else {
        on = fmaf(G.z, wy, -G.w * wx) > 0.f;
    }
    const float d = sqrtf(d2);
    return on ? -d : d;
}

// Record of an agent's off-road distance for the differentiable rollout:
// (segment << 3) | (corner << 1) | (1 if off road), -1 without a segment.
__device__ __forceinline__ int offroad_code(int e, int k, float sd) {
    return e >= 0 ? (e << 3) | (k << 1) | (sd > 0.f ? 1 : 0) : -1;
}

// The record of the corner holding the largest signed distance among the
// four lanes 4q .. 4q+3 (lane 4q+k: corner k), ties to the lower corner.
__device__ __forceinline__ int quad_argmax_code(float sd, int code, int lane) {
    int bk = lane & 3;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const float os = __shfl_xor_sync(kFull, sd, o);
        const int ok = __shfl_xor_sync(kFull, bk, o), oc = __shfl_xor_sync(kFull, code, o);
        if (os > sd || (os == sd && ok < bk)) {
            sd = os;
            bk = ok;
            code = oc;
        }
    }
    return code;
}

// REC: *orec (lane 0) receives the agent's offroad_code.
template <bool REC = false>
static __device__ float offroad_agent(const SegView& V, int lane, float xh, float xl, float yh, float yl, float c,
                                      float s, float hl, float hw, int32_t* hint, uint16_t* tl, float4* meta,
                                      Counts& cnt, bool force_scan = false, float lvx = 0.f, float lvy = 0.f,
                                      int32_t* orec = nullptr) {
    if (V.E == 0) {
        if (hint && lane < 4) hint[lane] = -1;
        if (REC && lane == 0) *orec = -1;
        return -WSIM_INF;
    }
    float cxl[4], cyl[4], px[4], py[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float a = (k < 2 ? 1.f : -1.f) * hl;
        const float b = (k == 0 || k == 3 ? 1.f : -1.f) * hw;
        cxl[k] = xl + fmaf(a, c, -b * s);
        cyl[k] = yl + fmaf(a, s, b * c);
        px[k] = xh + cxl[k];
        py[k] = yh + cyl[k];
    }
    // Upper bounds from the previous winners (lane k evaluates corner k).
    float dh = WSIM_INF;
    if (hint && lane < 4) {
        const int e = hint[lane];
        if (e >= 0 && e < V.E) dh = seg_dist2(V.geo[e], V.inv[e], xh, pick4(cxl, lane), yh, pick4(cyl, lane));
    }
    float u2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u2[k] = __shfl_sync(kFull, dh, k);
    if (!(u2[0] < WSIM_INF && u2[1] < WSIM_INF && u2[2] < WSIM_INF && u2[3] < WSIM_INF)) {
        // Bounds from points on segments (two per tile).
        float m[4] = {WSIM_INF, WSIM_INF, WSIM_INF, WSIM_INF};
        for (int t = lane; t < V.nt; t += 32) {
            const float4 P = V.tiles[2 * t];  // both chord ends lie on segments
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float ax = P.x - px[k], ay = P.y - py[k];
                const float bx = (P.x + P.z) - px[k], by = (P.y + P.w) - py[k];
                m[k] = fminf(m[k], fminf(fmaf(ax, ax, ay * ay), fmaf(bx, bx, by * by)));
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            m[k] = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(m[k])));
            u2[k] = fminf(u2[k], m[k]);
        }
        if (lane == 0) cnt.tiles += V.nt;
    }
    // Float32 corner positions in the box tests and bounds: 2 mm of slack.
    float lim2[4], ucap = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float u = sqrt_approx(u2[k]) * 1.000001f + 2e-3f;
        lim2[k] = u * u;
        ucap = fmaxf(ucap, u);
    }
    // Agent-level test: the centre's distance to a box or capsule minus the
    // half diagonal bounds every corner's distance to it from below.
    const float ccx = xh + xl, ccy = yh + yl;
    const float rad = sqrt_approx(fmaf(hl, hl, hw * hw)) * 1.000001f + 1e-3f;
    const float clim = (ucap + rad) * (ucap + rad);
    float lim[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) lim[k] = sqrt_approx(lim2[k]) * 1.000001f;

    float bd[4] = {WSIM_INF, WSIM_INF, WSIM_INF, WSIM_INF};
    int bi[4] = {-1, -1, -1, -1};
    bool done = false;
    if (tl && !force_scan) {
        // Cached candidate tiles: every tile whose box lies within radius r0
        // of centre c0.  A segment outside them is farther than
        // r0 - |p - c0| from corner p, so a best distance below that bound
        // is the exact nearest distance.
        const float4 M = *meta;
        const int n = __float_as_int(M.w);
        if (n >= 0) {
            unsigned cm = 0;
            int t = 0;
            if (lane < n) {
                t = tl[lane];
                const float4 C = V.tiles[2 * t];
                const float4 Q = V.tiles[2 * t + 1];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float l = lim[k] + Q.x;
                    if (cap_d2(C, Q.y, px[k], py[k]) <= l * l) cm |= 1u << k;
                }
            }
            if (lane == 0) cnt.tiles += n;
            unsigned want = __ballot_sync(kFull, cm != 0);
            while (want) scan_next_two(V, lane, want, t, cm, xh, yh, cxl, cyl, bd, bi, cnt);
            // best + |p - c0| <= r0 - 1 mm for every corner (approximate roots
            // rounded up); the reduced minima agree in all lanes.
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float b = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(bd[k])));
                const float dx = px[k] - M.x, dy = py[k] - M.y;
                ok = ok && (sqrt_approx(b) + sqrt_approx(fmaf(dx, dx, dy * dy))) * 1.000001f <= M.z - 1e-3f;
            }
            done = ok;
            if (!done) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    bd[k] = WSIM_INF;
                    bi[k] = -1;
                }
            }
        }
    }
    if (!done) {
        // Full search over the super-tiles; on the way, collect the next
        // candidate list.  Two lists are collected in one scan and the wider
        // is kept when it fits: the tiles within R of a centre moved ahead
        // of the agent by (lvx, lvy) (R grown by that distance, so the list
        // covers the agent's next steps), and the tiles within Rs of the
        // centre itself.
        const float dl = sqrt_approx(fmaf(lvx, lvx, lvy * lvy)) * 1.000001f;
        const float lcx = ccx + lvx, lcy = ccy + lvy;
        const float R = ucap + rad + kSkin + dl, Rs = ucap + rad + kSkinSmall;
        const float R2 = (R + 1e-3f) * (R + 1e-3f);
        const float slim = fmaxf(clim, (Rs + 1e-3f) * (Rs + 1e-3f));
        int nl = 0, nls = 0;
        int small_t = -1;  // the narrow list, entry n kept by lane n
        for (int sb = 0; sb < V.ns; sb += 32) {
            bool pass = false;
            if (sb + lane < V.ns) {
                const float4 B = V.sup[sb + lane];
                const float dx = fmaxf(fmaxf(B.x - ccx, ccx - B.z), 0.f);
                const float dy = fmaxf(fmaxf(B.y - ccy, ccy - B.w), 0.f);
                const float ex = fmaxf(fmaxf(B.x - lcx, lcx - B.z), 0.f);
                const float ey = fmaxf(fmaxf(B.y - lcy, lcy - B.w), 0.f);
                pass = fmaf(dx, dx, dy * dy) <= slim || fmaf(ex, ex, ey * ey) <= R2;
            }
            if (lane == 0) cnt.tiles += min(32, V.ns - sb);
            unsigned sup = __ballot_sync(kFull, pass);
            while (sup) {
                // Up to 32 / kSuper passing super-tiles at once, in index
                // order: lanes kSuper q .. kSuper q + kSuper-1 test the tiles
                // of the q-th, corner by corner (so tiles stay in increasing
                // order across lanes, and the lists too).
                unsigned rest = sup;
                for (int r = 0; r < lane / kSuper && rest; ++r) rest &= rest - 1;
                const int q = rest ? (sb + __ffs(rest) - 1) * kSuper + (lane & (kSuper - 1)) : V.nt;
                const int t = q < V.nt ? (V.perm ? static_cast<int>(V.perm[q]) : q) : V.nt;
                int taken = 0;
                for (; taken < 32 / kSuper && sup; ++taken) sup &= sup - 1;
                unsigned cm = 0;
                bool inl = false, inls = false;
                if (t < V.nt) {
                    const float4 C = V.tiles[2 * t];
                    const float4 Q = V.tiles[2 * t + 1];
                    const float dc = cap_d2(C, Q.y, ccx, ccy);
                    const float rl = R + Q.x + 1e-3f, rs = Rs + Q.x + 1e-3f, rc = ucap + rad + Q.x;
                    inl = cap_d2(C, Q.y, lcx, lcy) <= rl * rl;
                    inls = dc <= rs * rs;
                    if (dc <= rc * rc) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float l = lim[k] + Q.x;
                            if (cap_d2(C, Q.y, px[k], py[k]) <= l * l) cm |= 1u << k;
                        }
                    }
                }
                if (lane == 0) cnt.tiles += kSuper * taken;
                if (tl) {
                    const unsigned lb = __ballot_sync(kFull, inl);
                    const int pos = nl + __popc(lb & ((1u << lane) - 1u));
                    if (inl && pos < kList) tl[pos] = static_cast<uint16_t>(t);
                    nl += __popc(lb);
                    // narrow list: entry n is kept by lane n
                    unsigned sb2 = __ballot_sync(kFull, inls);
                    while (sb2) {
                        const int l = __ffs(sb2) - 1;
                        sb2 &= sb2 - 1;
                        const int tn = __shfl_sync(kFull, t, l);
                        if (lane == nls) small_t = tn;
                        ++nls;
                    }
                }
                unsigned want = __ballot_sync(kFull, cm != 0);
                while (want) scan_next_two<true>(V, lane, want, t, cm, xh, yh, cxl, cyl, bd, bi, cnt);
            }
        }
        if (tl) {
            // Lists are kept in increasing tile order (super-tiles come in
            // any order), so that their scans meet equal distances in
            // increasing index order.
            if (nl <= kList) {
                __syncwarp();
                const unsigned v = warp_sort_asc(lane < nl ? static_cast<unsigned>(tl[lane]) : 0xffffffffu, lane);
                __syncwarp();
                if (lane < nl) tl[lane] = static_cast<uint16_t>(v);
                if (lane == 0) *meta = make_float4(lcx, lcy, R, __int_as_float(nl));
            } else if (nls <= kList) {
                const unsigned v = warp_sort_asc(lane < nls ? static_cast<unsigned>(small_t) : 0xffffffffu, lane);
                __syncwarp();
                if (lane < nls) tl[lane] = static_cast<uint16_t>(v);
                if (lane == 0) *meta = make_float4(ccx, ccy, Rs, __int_as_float(nls));
            } else if (lane == 0) {
                *meta = make_float4(lcx, lcy, R, __int_as_float(-1));
            }
        }
    }
    // Nearest segment per corner: the lexicographic (distance, index)
    // minimum over lanes (distances >= 0 order like their bit patterns).
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned key = __float_as_uint(bd[k]);
        const unsigned mn = __reduce_min_sync(kFull, key);
        const unsigned id = __reduce_min_sync(kFull, key == mn ? static_cast<unsigned>(bi[k]) : 0xffffffffu);
        bd[k] = __uint_as_float(mn);
        bi[k] = static_cast<int>(id);
    }
    // Side of the nearest feature (lane k: corner k).
    float sd = -WSIM_INF;
    int code = -1;
    if (lane < 4) {
        const int e = pick4(bi, lane);
        if (e >= 0) sd = corner_side(V, e, pick4(bd, lane), xh, pick4(cxl, lane), yh, pick4(cyl, lane));
        if (hint) hint[lane] = e;
        if (REC) code = offroad_code(e, lane, sd);
    }
    if (REC) {
        code = quad_argmax_code(sd, code, lane);
        if (lane == 0) *orec = code;
    }
    sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 1));
    sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 2));
    return __shfl_sync(kFull, sd, 0);
}

// ---------------------------------------------------------------------------
// Off-road of eight agents (warp; lane 4a+k = corner k of agent a).  Fast
// path: the bound U from each corner's previous nearest segment, the
// agent's cached candidate tiles whose capsule lies within U (the agent's
// four lanes split the list and test each tile for all four corners), a
// scan of each corner's tiles, and the cache condition best + |p - c0| <=
// r0 - 1 mm (then the result is the exact nearest segment).  Agents whose cache or
// hints fail any corner take the warp-cooperative search (offroad_agent),
// which also rebuilds the cache.
// ---------------------------------------------------------------------------
// REC: orec[a] receives agent a's offroad_code.
template <bool REC = false>
static __device__ void offroad_group(AgentSmem& sm, const SegView& V, int32_t* hint_base, uint16_t* tl_base,
                                     float4* meta_base, int N, int g0, int lane, float look, Counts& cnt,
                                     int32_t* orec = nullptr) {
    const int a = g0 + (lane >> 2), k = lane & 3;
    const bool act = a < N && sm.valid[a];
    bool fast = false;
    float best = WSIM_INF;
    int bi = -1;
    float xh = 0.f, yh = 0.f, cl = 0.f, dl = 0.f, px = 0.f, py = 0.f;
    float4 M = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned mask = 0;
    const uint16_t* L = nullptr;
    float U = WSIM_INF;
    int n = -1;
    if (act && V.E > 0 && hint_base && tl_base) {
        const float hl = (k < 2 ? 1.f : -1.f) * sm.hl[a], hw = (k == 0 || k == 3 ? 1.f : -1.f) * sm.hw[a];
        const float c = sm.c[a], s = sm.s[a];
        xh = sm.xh[a];
        yh = sm.yh[a];
        cl = sm.xl[a] + fmaf(hl, c, -hw * s);
        dl = sm.yl[a] + fmaf(hl, s, hw * c);
        px = xh + cl;
        py = yh + dl;
        M = meta_base[a];
        n = __float_as_int(M.w);
        const int eh = hint_base[4 * a + k];
        if (n >= 0 && eh >= 0 && eh < V.E) {
            fast = true;
            U = sqrt_approx(seg_dist2(V.geo[eh], V.inv[eh], xh, cl, yh, dl)) * 1.000001f + 2e-3f;
        }
    }
    // The agent's four lanes split its list (lane k takes entries k, k+4,
    // ...) and test each tile against all four corners; the corner masks
    // are then gathered per lane.  Only agents whose four corners all have a
    // bound take the fast path.
    const unsigned qm = 0xfu << (lane & ~3);
    const bool qfast = (__ballot_sync(kFull, fast) & qm) == qm;
    float pxs[4], pys[4], us[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        pxs[c] = __shfl_sync(kFull, px, (lane & ~3) | c);
        pys[c] = __shfl_sync(kFull, py, (lane & ~3) | c);
        us[c] = __shfl_sync(kFull, U, (lane & ~3) | c);
    }
    unsigned mc[4] = {0u, 0u, 0u, 0u};
    if (qfast) {
        L = tl_base + kList * a;
        for (int j = k; j < n; j += 4) {
            const int t = L[j];
            const float4 C = V.tiles[2 * t];
            const float4 Q = V.tiles[2 * t + 1];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float l = us[c] + Q.x;
                if (cap_d2(C, Q.y, pxs[c], pys[c]) <= l * l) mc[c] |= 1u << j;
            }
        }
        cnt.tiles += n;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        unsigned v = mc[c];
        v |= __shfl_xor_sync(kFull, v, 1);
        v |= __shfl_xor_sync(kFull, v, 2);
        if (c == k) mask = v;
    }
    fast = qfast;
    // Scan each lane's passing tiles (lanes with fewer tiles idle).
    while (__any_sync(kFull, mask != 0)) {
        if (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1;
            const int e0 = static_cast<int>(L[j]) * kTile;
            cnt.evals += kTile;
            // every position of a tile holds a segment or far-away padding
            // (squared distance +inf, never the nearest)
#pragma unroll 8
            for (int q = 0; q < kTile; ++q) {
                const int e = e0 + q;
                const float d2 = seg_dist2(V.geo[e], V.inv[e], xh, cl, yh, dl);
                if (d2 < best) {
                    best = d2;
                    bi = e;
                }
            }
        }
    }
    bool ok = fast;
    if (fast) {
        const float dx = px - M.x, dy = py - M.y;
        ok = (sqrt_approx(best) + sqrt_approx(fmaf(dx, dx, dy * dy))) * 1.000001f <= M.z - 1e-3f;
    }
    // all four corners of the agent must pass
    unsigned okv = __ballot_sync(kFull, ok);
    const unsigned quad = 0xfu << (lane & ~3);
    ok = (okv & quad) == quad;
    float sd = -WSIM_INF;
    if (ok) {
        sd = corner_side(V, bi, best, xh, cl, yh, dl);
        hint_base[4 * a + k] = bi;
    }
    if (REC) {
        const int code = quad_argmax_code(sd, ok ? offroad_code(bi, k, sd) : -1, lane);
        if (ok && k == 0) orec[a] = code;
    }
    sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 1));
    sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 2));
    if (ok && k == 0) sm.off[a] = sd;
    // The others: warp-cooperative search (no usable cache or hint).
    unsigned need = __ballot_sync(kFull, act && !ok && k == 0);
    while (need) {
        const int ai = g0 + ((__ffs(need) - 1) >> 2);
        need &= need - 1;
        const float f = offroad_agent<REC>(V, lane, sm.xh[ai], sm.xl[ai], sm.yh[ai], sm.yl[ai], sm.c[ai], sm.s[ai],
                                           sm.hl[ai], sm.hw[ai], hint_base ? hint_base + 4 * ai : nullptr,
                                           tl_base ? tl_base + kList * ai : nullptr,
                                           tl_base ? meta_base + ai : nullptr, cnt, true, sm.vx[ai] * look,
                                           sm.vy[ai] * look, REC ? orec + ai : nullptr);
        if (lane == 0) sm.off[ai] = f;
    }
}

// ---------------------------------------------------------------------------
// Overlap rows (one warp per agent) and off-road (one warp per eight
// agents), both taken from shared counters.  sm.ov receives the row maxima;
// finish merges the columns.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void phase_metrics(AgentSmem& sm, const SegView& V, int32_t* hint_base, uint16_t* tl_base,
                              float4* meta_base, int N, bool do_ov, bool do_off, float look, Counts& cnt) {
    const int lane = threadIdx.x & 31;
    if (do_ov) {
        overlap_bounds<NT>(sm, N);
        __syncthreads();
        for (int i = next_agent(sm, 1, lane); i < N; i = next_agent(sm, 1, lane))
            if (sm.valid[i]) overlap_row(sm, N, i, lane, cnt);
    }
    if (do_off) {
        for (int g = next_agent(sm, 2, lane); 8 * g < N; g = next_agent(sm, 2, lane))
            offroad_group(sm, V, hint_base, tl_base, meta_base, N, 8 * g, lane, look, cnt);
    }
}

// The warp tasks of the metrics: off-road groups from work[2], and overlap
// rows from work[1] (with the overlap culling records already in place).
__device__ __forceinline__ void offroad_tasks(AgentSmem& sm, const SegView& V, int32_t* hint_base, uint16_t* tl_base,
                                              float4* meta_base, int N, float look, Counts& cnt) {
    const int lane = threadIdx.x & 31;
    for (int g = next_agent(sm, 2, lane); 8 * g < N; g = next_agent(sm, 2, lane))
        offroad_group(sm, V, hint_base, tl_base, meta_base, N, 8 * g, lane, look, cnt);
}
// Rows q and N-1-q of the pair triangle as one warp task of the
// scene-resident rollout: N-1 pairs for every q, so the lanes stay full
// (single rows left a quarter of the lanes idle on average); an invalid
// agent's record fails every bound test, as an absent partner's does.  The
// same pairs and maxima as overlap_row (max is order-free).
static __device__ void overlap_rows2(AgentSmem& sm, int N, int q, int lane, Counts& cnt) {
    const int ia = q, ib = N - 1 - q;
    const int na = N - 1 - ia, nb = ib > ia ? N - 1 - ib : 0;
    for (int u = lane; u < na + nb; u += 32) {
        const bool in_a = u < na;
        const int i = in_a ? ia : ib;
        const int j = in_a ? ia + 1 + u : ib + 1 + (u - na);
        const float4 Pi = sm.obox[i];
        const float4 Pj = sm.obox[j];  // invalid agents: R = -inf, always skipped
        cnt.bounds += 1;
        const float dx = Pj.x - Pi.x, dy = Pj.y - Pi.y;
        const float t = fmaxf(Pi.w + Pj.z, Pi.z + Pj.w);  // |dc| / sqrt(2) above this: skip
        if (!(t >= 0.f) || fmaf(dx, dx, dy * dy) > 2.f * t * t) continue;
        const float ddx = comp_diff(sm.xh[j], sm.xl[j], sm.xh[i], sm.xl[i]);
        const float ddy = comp_diff(sm.yh[j], sm.yl[j], sm.yh[i], sm.yl[i]);
        const float d = sat_depth(ddx, ddy, sm.c[i], sm.s[i], sm.hl[i], sm.hw[i], sm.c[j], sm.s[j], sm.hl[j], sm.hw[j]);
        atomicMax(&sm.ovk[j], ukey(d));
        atomicMax(&sm.pk[j], partner_key(d, i));
        atomicMax(&sm.ovk[i], ukey(d));
        atomicMax(&sm.pk[i], partner_key(d, j));
        cnt.pairs += 2;
    }
}

__device__ __forceinline__ void row_tasks(AgentSmem& sm, int N, Counts& cnt) {
    const int lane = threadIdx.x & 31;
    for (int q = next_agent(sm, 1, lane); 2 * q < N; q = next_agent(sm, 1, lane)) overlap_rows2(sm, N, q, lane, cnt);
}

// ov_i of a valid agent after phase_metrics.
__device__ __forceinline__ float merged_ov(const AgentSmem& sm, int i) { return unukey(sm.ovk[i]); }

// ---------------------------------------------------------------------------
// Log divergence, flags, metric stores and the scene reward.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void phase_finish(AgentSmem& sm, const StepArgs& A, const MetricsP& m, int32_t* reward, int t_log, int a0,
                             int N) {
    if (threadIdx.x == 0) sm.reward = 0;
    __syncthreads();
    int r = 0;
    for (int i = threadIdx.x; i < N; i += NT) {
        const int g = a0 + i;
        float ov = 0.f, off = 0.f, ld = 0.f;
        uint8_t fl = 0;
        if (sm.valid[i]) {
            const size_t li = static_cast<size_t>(t_log) * A.N_tot + g;
            const float dx = (sm.xh[i] - A.log_x[li]) + sm.xl[i];
            const float dy = (sm.yh[i] - A.log_y[li]) + sm.yl[i];
            ld = sqrtf(fmaf(dx, dx, dy * dy));
            ov = merged_ov(sm, i);
            off = sm.off[i];
            fl = (ov > 0.f ? WSIM_FLAG_COLLISION : 0) | (off > 0.f ? WSIM_FLAG_OFFROAD : 0) |
                 (sm.kin[i] ? WSIM_FLAG_KININF : 0);
            r -= (ov > 0.f) + (off > 0.f);
        }
        m.ov[g] = ov;
        m.off[g] = off;
        m.logdiv[g] = ld;
        m.flags[g] = fl;
    }
    if (r) atomicAdd(&sm.reward, r);
    __syncthreads();
    if (threadIdx.x == 0) *reward = sm.reward;
}

// ---------------------------------------------------------------------------
// The per-agent phase of the pipelined rollout step (thread per agent, between
// two barriers).  For agent i, in this order: (1) finish the metrics of the
// current state (log row t_log; metric row m; the scene's reward summed into
// sm.reward); (2) advance to the next state (n* -> current, the
// kinematic-infeasibility flag of that transition, the state stored to out,
// the cos / sin of its heading); then, after a barrier, (3) prepare the
// overlap culling record of the next state from the current arrays (the
// partner's heading cos / sin is not computed a second time) and clear the
// overlap maxima.  Before the barrier every read of another agent's data is
// of arrays the pass does not write.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void finish_advance(AgentSmem& sm, const StepArgs& A, const MetricsP* m, int t_log, bool advance,
                               const StateP* out, int a0, int N) {
    const Params& p = A.p;
    int r = 0;
    for (int i = threadIdx.x; i < N; i += NT) {
        const int g = a0 + i;
        if (m) {
            float ov = 0.f, off = 0.f, ld = 0.f;
            uint8_t fl = 0;
            if (sm.valid[i]) {
                const size_t li = static_cast<size_t>(t_log) * A.N_tot + g;
                const float dx = (sm.xh[i] - A.log_x[li]) + sm.xl[i];
                const float dy = (sm.yh[i] - A.log_y[li]) + sm.yl[i];
                ld = sqrtf(fmaf(dx, dx, dy * dy));
                ov = merged_ov(sm, i);
                off = sm.off[i];
                fl = (ov > 0.f ? WSIM_FLAG_COLLISION : 0) | (off > 0.f ? WSIM_FLAG_OFFROAD : 0) |
                     (sm.kin[i] ? WSIM_FLAG_KININF : 0);
                r -= (ov > 0.f) + (off > 0.f);
            }
            m->ov[g] = ov;
            m->off[g] = off;
            m->logdiv[g] = ld;
            m->flags[g] = fl;
        }
        if (!advance) continue;
        sm.kin[i] = sm.valid[i] ? kin_infeasible(p, sm.vx[i], sm.vy[i], sm.thh[i], sm.thl[i], sm.nvx[i], sm.nvy[i])
                                : uint8_t(0);
        if (out) {
            out->x[g] = sm.nxh[i];
            out->x_lo[g] = sm.nxl[i];
            out->y[g] = sm.nyh[i];
            out->y_lo[g] = sm.nyl[i];
            out->th[g] = sm.nth[i];
            out->th_lo[g] = sm.ntl[i];
            out->vx[g] = sm.nvx[i];
            out->vy[g] = sm.nvy[i];
            out->s[g] = sm.nsh[i];
            out->s_lo[g] = sm.nsl[i];
        }
        sm.xh[i] = sm.nxh[i];
        sm.xl[i] = sm.nxl[i];
        sm.yh[i] = sm.nyh[i];
        sm.yl[i] = sm.nyl[i];
        sm.thh[i] = sm.nth[i];
        sm.thl[i] = sm.ntl[i];
        float c, s;
        comp_sincos(sm.nth[i], sm.ntl[i], c, s);
        sm.c[i] = c;
        sm.s[i] = s;
        sm.vx[i] = sm.nvx[i];
        sm.vy[i] = sm.nvy[i];
        sm.sh[i] = sm.nsh[i];
        sm.sl[i] = sm.nsl[i];
    }
    if (r) atomicAdd(&sm.reward, r);
    if (threadIdx.x == 0) sm.work[0] = sm.work[1] = sm.work[2] = 0;  // the next task phase
    if (!advance) return;
    // Overlap culling record of the new state, once every agent's new state
    // (and its heading's cos / sin) is in the current arrays: the depth
    // against the deepest partner of the step just measured, a lower bound
    // of the new maximum; then the maxima are cleared.
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += NT) {
        float lb = -WSIM_INF;
        const int q = (sm.pk[i] >> 8) > (kNoDepth >> 8) ? static_cast<int>(sm.pk[i] & 0xffu) : -1;
        if (sm.valid[i] && q >= 0 && q < N && q != i && sm.valid[q]) {
            const int a = min(i, q), b = max(i, q);
            const float dx = comp_diff(sm.xh[b], sm.xl[b], sm.xh[a], sm.xl[a]);
            const float dy = comp_diff(sm.yh[b], sm.yl[b], sm.yh[a], sm.yl[a]);
            lb = sat_depth(dx, dy, sm.c[a], sm.s[a], sm.hl[a], sm.hw[a], sm.c[b], sm.s[b], sm.hl[b], sm.hw[b]);
        }
        const float R = (sm.hl[i] + sm.hw[i]) * 1.000001f + 5e-4f;
        sm.obox[i] = sm.valid[i] ? make_float4(sm.xh[i], sm.yh[i], R, R - lb + 5e-4f)
                                 : make_float4(sm.xh[i], sm.yh[i], -WSIM_INF, -WSIM_INF);
        sm.ovk[i] = kNoDepth;
        sm.pk[i] = kNoDepth;
    }
}

// ---------------------------------------------------------------------------
// CTA setup and counters.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void init_cta(AgentSmem& sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        for (int k = 0; k < kCounters; ++k) sm.cnt[k] = 0;
    }
    __syncthreads();
}

__device__ __forceinline__ void publish_counts(AgentSmem& sm, const StepArgs& A, const Counts& c) {
    if (A.count) {
        const uint32_t v[kCounters] = {c.evals, c.tiles, c.pairs, c.tests, c.bounds, c.filters};
#pragma unroll
        for (int k = 0; k < kCounters; ++k)
            if (v[k]) atomicAdd(&sm.cnt[k], static_cast<unsigned long long>(v[k]));
    }
    __syncthreads();
    if (A.count && threadIdx.x == 0)
        for (int k = 0; k < kCounters; ++k)
            if (sm.cnt[k]) atomicAdd(&A.counters[k], sm.cnt[k]);
}

// Scene s's segments in global memory.
__device__ __forceinline__ SegView global_view(const Segs& G, int s) {
    const int e0 = G.off[s];
    const int E = G.cnt[s];
    const int nt = (E + kTile - 1) / kTile;
    return SegView{G.geo + e0, G.inv + e0, G.flags + e0, G.tiles + 2 * (e0 / kTile), G.sup + G.soff[s],
                   E, nt, (nt + kSuper - 1) / kSuper, G.tperm ? G.tperm + e0 / kTile : nullptr};
}

}  // namespace wsim
