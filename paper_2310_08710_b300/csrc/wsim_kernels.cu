// wsim step kernels for sm_103a.
//
// One CTA owns one scene at a time.  The fused step kernel is persistent: its
// CTAs take scene ids from an atomic work counter over a cost-ordered list,
// so scenes of uneven size share one launch.  Per scene it runs
//   transition  (Sec. 4 step): IDM agents warp-cooperatively (one look-ahead
//               sample per lane, Sec. 3.5), policy agents one per thread
//               (bicycle / delta dynamics, App. A.1), compensated positions;
//   overlap     (Sec. 3.4 collision): all pairs from shared-memory boxes,
//               one warp per agent, warp max-reduction;
//   off-road    (Sec. 3.4 off-road): every box corner against every road-edge
//               segment of the scene, segments streamed through shared memory
//               in chunks by bulk async copies (TMA) on a two-stage mbarrier
//               pipeline;
//   finish      log divergence (Sec. 3.4), flags and the sparse reward
//               (Sec. 5.2).
// The plain path runs the same phases as separate one-CTA launches per scene.
#include <math_constants.h>

#include "wsim_device.cuh"

namespace wsim {

#define kInf CUDART_INF_F
constexpr unsigned kFull = 0xffffffffu;

struct __align__(16) Smem {
    float4 geo[2][kChunk];
    float inv[2][kChunk];
    uint64_t bar[2];
    // boxes of the state being read (t during the transition, t+1 after)
    float xh[kMaxN], xl[kMaxN], yh[kMaxN], yl[kMaxN], c[kMaxN], s[kMaxN], hl[kMaxN], hw[kMaxN];
    float vx[kMaxN], vy[kMaxN];
    // next state
    float nxh[kMaxN], nxl[kMaxN], nyh[kMaxN], nyl[kMaxN], nth[kMaxN], ntl[kMaxN];
    float nvx[kMaxN], nvy[kMaxN], nsh[kMaxN], nsl[kMaxN];
    float ov[kMaxN], off[kMaxN];
    uint8_t valid[kMaxN];
    int scene;
    int reward;
    unsigned long long cnt[4];
};

// ---------------------------------------------------------------------------
// Loading and storing agent state.
// ---------------------------------------------------------------------------
__device__ void load_boxes(Smem& sm, const StepArgs& A, const CStateP& st, int a0, int N) {
    for (int i = threadIdx.x; i < N; i += kThreads) {
        const int g = a0 + i;
        sm.xh[i] = st.x[g];
        sm.xl[i] = st.x_lo[g];
        sm.yh[i] = st.y[g];
        sm.yl[i] = st.y_lo[g];
        float c, s;
        comp_sincos(st.th[g], st.th_lo[g], c, s);
        sm.c[i] = c;
        sm.s[i] = s;
        sm.hl[i] = 0.5f * A.L[g];
        sm.hw[i] = 0.5f * A.W[g];
        sm.vx[i] = st.vx[g];
        sm.vy[i] = st.vy[g];
        sm.valid[i] = A.valid[g];
    }
}

// Write the next state to global memory and make it the current box set.
__device__ void writeback(Smem& sm, const StepArgs& A, int a0, int N) {
    for (int i = threadIdx.x; i < N; i += kThreads) {
        const int g = a0 + i;
        A.out.x[g] = sm.nxh[i];
        A.out.x_lo[g] = sm.nxl[i];
        A.out.y[g] = sm.nyh[i];
        A.out.y_lo[g] = sm.nyl[i];
        A.out.th[g] = sm.nth[i];
        A.out.th_lo[g] = sm.ntl[i];
        A.out.vx[g] = sm.nvx[i];
        A.out.vy[g] = sm.nvy[i];
        A.out.s[g] = sm.nsh[i];
        A.out.s_lo[g] = sm.nsl[i];
        sm.xh[i] = sm.nxh[i];
        sm.xl[i] = sm.nxl[i];
        sm.yh[i] = sm.nyh[i];
        sm.yl[i] = sm.nyl[i];
        float c, s;
        comp_sincos(sm.nth[i], sm.ntl[i], c, s);
        sm.c[i] = c;
        sm.s[i] = s;
        sm.vx[i] = sm.nvx[i];
        sm.vy[i] = sm.nvy[i];
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
// IDM route following of agent i (Sec. 3.5; textbook IDM of Treiber et al.).
// Warp-cooperative: lane k holds look-ahead sample k+1 at route parameter
// s + L/2 + dq (k+1).  For every other valid agent j the warp tests all 32
// samples against j's box widened by half this agent's width; the ballot's
// lowest set bit is the first hit.  The lead is the hit agent with the
// smallest bumper gap (ties: lower index).
// ---------------------------------------------------------------------------
__device__ void idm_agent(Smem& sm, const StepArgs& A, int a0, int N, int i, int lane,
                          unsigned long long& n_tests) {
    const Params& p = A.p;
    const int g = a0 + i;
    const int ro = A.route_off[g];
    const int P = A.route_off[g + 1] - ro;
    const float* rx = A.route_x + ro;
    const float* ry = A.route_y + ro;
    const float s_hi = A.in.s[g], s_lo = A.in.s_lo[g];
    const float vxi = sm.vx[i], vyi = sm.vy[i];
    const float v = sqrtf(fmaf(vxi, vxi, vyi * vyi));
    const float hli = sm.hl[i], wi = sm.hw[i];

    // This lane's look-ahead sample.
    float bh, bl;
    two_sum(s_hi, fmaf(p.dq, static_cast<float>(lane + 1), hli), bh, bl);
    bl = __fadd_rn(bl, s_lo);
    int seg;
    float tau;
    route_locate(bh, bl, p, P, seg, tau);
    const float Px = rx[seg], Py = ry[seg];
    const float dx = rx[seg + 1] - Px, dy = ry[seg + 1] - Py;
    const float qox = tau * dx, qoy = tau * dy;
    const float rn = rsqrtf(fmaf(dx, dx, dy * dy));
    const float tx = dx * rn, ty = dy * rn;

    // Bounding circle of the samples (prefilter of far agents).
    const float qx = Px + qox, qy = Py + qoy;
    const float cx = __shfl_sync(kFull, qx, 15), cy = __shfl_sync(kFull, qy, 15);
    float rq = sqrtf((qx - cx) * (qx - cx) + (qy - cy) * (qy - cy));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rq = fmaxf(rq, __shfl_xor_sync(kFull, rq, o));

    const float xih = sm.xh[i], xil = sm.xl[i], yih = sm.yh[i], yil = sm.yl[i];
    int lead = -1, lead_hit = 0;
    float gbest = kInf;
    for (int j = 0; j < N; ++j) {
        if (j == i || !sm.valid[j]) continue;
        const float xjh = sm.xh[j], yjh = sm.yh[j];
        const float hlj = sm.hl[j], hwj = sm.hw[j];
        const float ex = xjh - cx, ey = yjh - cy;
        const float reach = rq + hlj + hwj + 2.f * wi + 0.05f;
        if (ex * ex + ey * ey > reach * reach) continue;
        if (lane == 0) n_tests += 32;
        const float rxq = (Px - xjh) + (qox - sm.xl[j]);
        const float ryq = (Py - yjh) + (qoy - sm.yl[j]);
        const float cj = sm.c[j], sj = sm.s[j];
        const float pu = fabsf(fmaf(rxq, cj, ryq * sj));
        const float pn = fabsf(fmaf(-rxq, sj, ryq * cj));
        const float m = fminf(hlj + wi - pu, hwj + wi - pn);
        const unsigned hits = __ballot_sync(kFull, m >= 0.f);
        if (!hits) continue;
        const float ddx = comp_diff(xjh, sm.xl[j], xih, xil);
        const float ddy = comp_diff(yjh, sm.yl[j], yih, yil);
        const float gap = fmaxf(p.gap_min, sqrtf(fmaf(ddx, ddx, ddy * ddy)) - (hli + hlj));
        if (gap < gbest) {
            gbest = gap;
            lead = j;
            lead_hit = __ffs(hits) - 1;
        }
    }

    // IDM acceleration (exponent 4).
    const float r = v / A.v0[g];
    const float r2 = r * r;
    const float r4 = r2 * r2;
    float acc;
    if (lead >= 0) {
        const float tlx = __shfl_sync(kFull, tx, lead_hit);
        const float tly = __shfl_sync(kFull, ty, lead_hit);
        const float vl = fmaf(sm.vx[lead], tlx, sm.vy[lead] * tly);
        const float sstar = p.s0 + fmaxf(0.f, fmaf(v, p.T, v * (v - vl) / p.idm_sqrt_ab2));
        const float q = sstar / gbest;
        acc = p.amax * (1.f - r4 - q * q);
    } else {
        acc = p.amax * (1.f - r4);
    }
    // Advance along the route by the trapezoidal distance of the new speed.
    const float vn = fmaxf(0.f, fmaf(acc, p.dt, v));
    float sh = s_hi, sl = s_lo;
    comp_add(sh, sl, 0.5f * (v + vn) * p.dt);
    int sg;
    float ta;
    route_locate(sh, sl, p, P, sg, ta);
    const float Qx = rx[sg], Qy = ry[sg];
    const float ux = rx[sg + 1] - Qx, uy = ry[sg + 1] - Qy;
    if (lane == 0) {
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
}

// ---------------------------------------------------------------------------
// Transition t -> t+1 of one scene into the n* arrays.
// ---------------------------------------------------------------------------
__device__ void phase_transition(Smem& sm, const StepArgs& A, int a0, int N, unsigned long long& n_tests) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < N; i += kWarps) {
        if (A.kind[a0 + i] == WSIM_KIND_IDM && sm.valid[i]) idm_agent(sm, A, a0, N, i, lane, n_tests);
    }
    const Params& p = A.p;
    for (int i = threadIdx.x; i < N; i += kThreads) {
        const int g = a0 + i;
        const int kind = A.kind[g];
        if (kind == WSIM_KIND_IDM && sm.valid[i]) continue;
        float xh = sm.xh[i], xl = sm.xl[i], yh = sm.yh[i], yl = sm.yl[i];
        float thh = A.in.th[g], thl = A.in.th_lo[g];
        float vx = sm.vx[i], vy = sm.vy[i];
        const bool moves = sm.valid[i] && kind != WSIM_KIND_IDM && (A.ctrl == nullptr || A.ctrl[g]);
        if (moves && kind == WSIM_KIND_BICYCLE) {
            // App. A.1 bicycle forward dynamics.
            const float a = A.act[g], k = A.act[A.N_tot + g];
            if (!isfinite(a) || !isfinite(k)) set_status(A.status, WSIM_ENONFINITE);
            const float v = sqrtf(fmaf(vx, vx, vy * vy));
            const float hdt2 = 0.5f * p.dt * p.dt;
            const float ah = a * hdt2;
            comp_add(xh, xl, fmaf(vx, p.dt, ah * sm.c[i]));
            comp_add(yh, yl, fmaf(vy, p.dt, ah * sm.s[i]));
            comp_add(thh, thl, k * fmaf(v, p.dt, ah));
            const float vn = fmaf(a, p.dt, v);
            float cn, sn;
            comp_sincos(thh, thl, cn, sn);
            vx = vn * cn;
            vy = vn * sn;
        } else if (moves && kind == WSIM_KIND_DELTA) {
            // App. A.1 delta dynamics.
            const float ddx = A.act[g], ddy = A.act[A.N_tot + g], dth = A.act[2 * A.N_tot + g];
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
        sm.nsh[i] = A.in.s[g];
        sm.nsl[i] = A.in.s_lo[g];
    }
}

// ---------------------------------------------------------------------------
// Overlap: ov_i = max over valid j != i of the SAT depth d_ij, computed in the
// canonical order (min(i,j), max(i,j)) so that d_ij == d_ji bit for bit.
// ---------------------------------------------------------------------------
__device__ void phase_overlap(Smem& sm, int N, unsigned long long& n_pairs) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < N; i += kWarps) {
        float best = -kInf;
        if (sm.valid[i]) {
            for (int j = lane; j < N; j += 32) {
                if (j == i || !sm.valid[j]) continue;
                const int lo = min(i, j), hi = max(i, j);
                const float dx = comp_diff(sm.xh[hi], sm.xl[hi], sm.xh[lo], sm.xl[lo]);
                const float dy = comp_diff(sm.yh[hi], sm.yl[hi], sm.yh[lo], sm.yl[lo]);
                best = fmaxf(best, sat_depth(dx, dy, sm.c[lo], sm.s[lo], sm.hl[lo], sm.hw[lo], sm.c[hi], sm.s[hi],
                                             sm.hl[hi], sm.hw[hi]));
                ++n_pairs;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(kFull, best, o));
        }
        if (lane == 0) sm.ov[i] = best;
    }
}

// ---------------------------------------------------------------------------
// Off-road: signed distance of each box corner to its nearest road-edge
// segment.  Corner q = 4 i + c of agent i sits in thread q mod kThreads,
// slot q / kThreads.  Segments arrive in chunks of kChunk via bulk copies,
// double-buffered; every thread scans the whole chunk from shared memory
// (broadcast reads).  Returns false if a copy did not complete in time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void issue_chunk(Smem& sm, const StepArgs& A, int e0, int E, int c, int b) {
    const int n = min(kChunk, E - c * kChunk);
    const int np = (n + kSegAlign - 1) & ~(kSegAlign - 1);
    const uint32_t gb = static_cast<uint32_t>(np) * 16u, ib = static_cast<uint32_t>(np) * 4u;
    fence_proxy_async();
    mbar_expect_tx(&sm.bar[b], gb + ib);
    bulk_g2s(&sm.geo[b][0], A.segs.geo + e0 + c * kChunk, gb, &sm.bar[b]);
    bulk_g2s(&sm.inv[b][0], A.segs.inv + e0 + c * kChunk, ib, &sm.bar[b]);
}

// `phase` holds the parity each barrier waits for next (bit b for bar[b]).
__device__ bool phase_offroad(Smem& sm, const StepArgs& A, int s, int N, uint32_t& phase,
                              unsigned long long& n_evals) {
    const int tid = threadIdx.x;
    const int e0 = A.segs.off[s], E = A.segs.cnt[s];
    const int nq = 4 * N;
    const int R = (nq + kThreads - 1) / kThreads;
    float cxh[4], cxl[4], cyh[4], cyl[4], bd[4];
    int bi[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = tid + r * kThreads;
        bd[r] = kInf;
        bi[r] = -1;
        cxh[r] = cxl[r] = cyh[r] = cyl[r] = 0.f;
        if (r < R && q < nq) {
            const int i = q >> 2, c = q & 3;
            const float sl = c < 2 ? 1.f : -1.f;
            const float sw = (c == 0 || c == 3) ? 1.f : -1.f;
            const float hl = sl * sm.hl[i], hw = sw * sm.hw[i];
            cxh[r] = sm.xh[i];
            cyh[r] = sm.yh[i];
            cxl[r] = sm.xl[i] + fmaf(hl, sm.c[i], -hw * sm.s[i]);
            cyl[r] = sm.yl[i] + fmaf(hl, sm.s[i], hw * sm.c[i]);
        }
    }
    const int nch = (E + kChunk - 1) / kChunk;
    if (tid == 0) {
        for (int c = 0; c < nch && c < 2; ++c) issue_chunk(sm, A, e0, E, c, c);
    }
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        const uint32_t par = (phase >> b) & 1u;
        const bool ok = mbar_wait_bounded(&sm.bar[b], par, kWaitLimitNs);
        phase ^= 1u << b;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) set_status(A.status, WSIM_ETIMEOUT);
            // Give the copies still in flight (this chunk's and the next
            // one's) a bounded chance to land before the CTA leaves.
            mbar_wait_bounded(&sm.bar[b], par, kWaitLimitNs);
            if (c + 1 < nch) mbar_wait_bounded(&sm.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, kWaitLimitNs);
            __syncthreads();
            return false;
        }
        const int n = min(kChunk, E - c * kChunk);
        const int base = c * kChunk;
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            const float4 G = sm.geo[b][j];
            const float iv = sm.inv[b][j];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < R) {
                    const float wx = (cxh[r] - G.x) + cxl[r];
                    const float wy = (cyh[r] - G.y) + cyl[r];
                    const float t = __saturatef(fmaf(wx, G.z, wy * G.w) * iv);
                    const float ex = fmaf(-t, G.z, wx), ey = fmaf(-t, G.w, wy);
                    const float d2 = fmaf(ex, ex, ey * ey);
                    if (d2 < bd[r]) {
                        bd[r] = d2;
                        bi[r] = base + j;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && c + 2 < nch) issue_chunk(sm, A, e0, E, c + 2, b);
    }
    if (tid == 0) n_evals += static_cast<unsigned long long>(nq) * static_cast<unsigned long long>(E);

    // Side of the nearest feature; vertex rule where the nearest point is a
    // vertex shared by two segments.
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (r >= R) continue;
        const int q = tid + r * kThreads;
        float sd = -kInf;
        if (q < nq && bi[r] >= 0) {
            const int e = e0 + bi[r];
            const float4 G = A.segs.geo[e];
            const uint8_t fl = A.segs.flags[e];
            const float wx = (cxh[r] - G.x) + cxl[r];
            const float wy = (cyh[r] - G.y) + cyl[r];
            const float traw = fmaf(wx, G.z, wy * G.w) * A.segs.inv[e];
            bool on;
            if (traw <= 0.f && (fl & 1)) {
                const float4 Gp = A.segs.geo[e - 1];
                const bool l1 = fmaf(Gp.z, wy, -Gp.w * wx) > 0.f;
                const bool l2 = fmaf(G.z, wy, -G.w * wx) > 0.f;
                const float turn = fmaf(Gp.z, G.w, -Gp.w * G.z);
                on = turn > 0.f ? (l1 && l2) : (turn < 0.f ? (l1 || l2) : l1);
            } else if (traw >= 1.f && (fl & 2)) {
                const float4 Gn = A.segs.geo[e + 1];
                const float px = wx - G.z, py = wy - G.w;
                const bool l1 = fmaf(G.z, py, -G.w * px) > 0.f;
                const bool l2 = fmaf(Gn.z, py, -Gn.w * px) > 0.f;
                const float turn = fmaf(G.z, Gn.w, -G.w * Gn.z);
                on = turn > 0.f ? (l1 && l2) : (turn < 0.f ? (l1 || l2) : l1);
            } else {
                on = fmaf(G.z, wy, -G.w * wx) > 0.f;
            }
            const float d = sqrtf(bd[r]);
            sd = on ? -d : d;
        }
        // off_i = max over the agent's four corners (lanes 4m .. 4m+3).
        sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 1));
        sd = fmaxf(sd, __shfl_xor_sync(kFull, sd, 2));
        if ((tid & 3) == 0 && q < nq) sm.off[q >> 2] = sd;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Log divergence, flags, metric stores and the scene reward.
// ---------------------------------------------------------------------------
__device__ void phase_finish(Smem& sm, const StepArgs& A, int s, int a0, int N) {
    if (threadIdx.x == 0) sm.reward = 0;
    __syncthreads();
    int r = 0;
    for (int i = threadIdx.x; i < N; i += kThreads) {
        const int g = a0 + i;
        float ov = 0.f, off = 0.f, ld = 0.f;
        uint8_t fl = 0;
        if (sm.valid[i]) {
            const size_t li = static_cast<size_t>(A.t_log) * A.N_tot + g;
            const float dx = (sm.xh[i] - A.log_x[li]) + sm.xl[i];
            const float dy = (sm.yh[i] - A.log_y[li]) + sm.yl[i];
            ld = sqrtf(fmaf(dx, dx, dy * dy));
            ov = sm.ov[i];
            off = sm.off[i];
            fl = (ov > 0.f ? WSIM_FLAG_COLLISION : 0) | (off > 0.f ? WSIM_FLAG_OFFROAD : 0);
            r -= (ov > 0.f) + (off > 0.f);
        }
        A.m.ov[g] = ov;
        A.m.off[g] = off;
        A.m.logdiv[g] = ld;
        A.m.flags[g] = fl;
    }
    if (r) atomicAdd(&sm.reward, r);
    __syncthreads();
    if (threadIdx.x == 0) A.m.reward[s] = sm.reward;
}

__device__ void flush_counts(Smem& sm, const StepArgs& A, unsigned long long a, unsigned long long b,
                             unsigned long long c) {
    if (!A.count) return;
    if (a) atomicAdd(&sm.cnt[0], a);
    if (b) atomicAdd(&sm.cnt[2], b);
    if (c) atomicAdd(&sm.cnt[3], c);
}

__device__ void init_cta(Smem& sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        for (int k = 0; k < 4; ++k) sm.cnt[k] = 0;
    }
    __syncthreads();
}

__device__ void publish_counts(Smem& sm, const StepArgs& A) {
    __syncthreads();
    if (A.count && threadIdx.x == 0)
        for (int k = 0; k < 4; ++k)
            if (sm.cnt[k]) atomicAdd(&A.counters[k], sm.cnt[k]);
}

// ---------------------------------------------------------------------------
// Fused persistent step (or metrics-only) kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_step(const StepArgs A) {
    __shared__ Smem sm;
    init_cta(sm);
    uint32_t phase = 0u;
    unsigned long long n_evals = 0, n_pairs = 0, n_tests = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.scene = atomicAdd(A.queue, 1);
        __syncthreads();
        const int w = sm.scene;
        if (w >= A.S) break;
        const int s = A.order[w];
        const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
        load_boxes(sm, A, A.in, a0, N);
        __syncthreads();
        if (A.do_transition) {
            phase_transition(sm, A, a0, N, n_tests);
            __syncthreads();
            writeback(sm, A, a0, N);
            __syncthreads();
        }
        if (A.do_metrics) {
            phase_overlap(sm, N, n_pairs);
            if (!phase_offroad(sm, A, s, N, phase, n_evals)) break;
            __syncthreads();
            phase_finish(sm, A, s, a0, N);
        }
        __syncthreads();
    }
    flush_counts(sm, A, n_evals, n_pairs, n_tests);
    publish_counts(sm, A);
}

// ---------------------------------------------------------------------------
// Plain path: one single-CTA launch per scene and phase.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_plain_transition(const StepArgs A, int s) {
    __shared__ Smem sm;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    unsigned long long n_tests = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) sm.cnt[k] = 0;
    load_boxes(sm, A, A.in, a0, N);
    __syncthreads();
    phase_transition(sm, A, a0, N, n_tests);
    __syncthreads();
    writeback(sm, A, a0, N);
    flush_counts(sm, A, 0, 0, n_tests);
    publish_counts(sm, A);
}

__device__ CStateP as_const(const StateP& s) {
    return CStateP{s.x, s.y, s.x_lo, s.y_lo, s.th, s.th_lo, s.vx, s.vy, s.s, s.s_lo};
}

__global__ void __launch_bounds__(kThreads) k_plain_overlap(const StepArgs A, int s) {
    __shared__ Smem sm;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    unsigned long long n_pairs = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) sm.cnt[k] = 0;
    load_boxes(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    __syncthreads();
    phase_overlap(sm, N, n_pairs);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += kThreads) A.m.ov[a0 + i] = sm.ov[i];
    flush_counts(sm, A, 0, n_pairs, 0);
    publish_counts(sm, A);
}

__global__ void __launch_bounds__(kThreads) k_plain_offroad(const StepArgs A, int s) {
    __shared__ Smem sm;
    init_cta(sm);
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    uint32_t phase = 0u;
    unsigned long long n_evals = 0;
    load_boxes(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    __syncthreads();
    if (phase_offroad(sm, A, s, N, phase, n_evals)) {
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += kThreads) A.m.off[a0 + i] = sm.off[i];
    }
    flush_counts(sm, A, n_evals, 0, 0);
    publish_counts(sm, A);
}

__global__ void __launch_bounds__(kThreads) k_plain_finish(const StepArgs A, int s) {
    __shared__ Smem sm;
    const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
    load_boxes(sm, A, A.do_transition ? as_const(A.out) : A.in, a0, N);
    for (int i = threadIdx.x; i < N; i += kThreads) {
        sm.ov[i] = A.m.ov[a0 + i];
        sm.off[i] = A.m.off[a0 + i];
    }
    __syncthreads();
    phase_finish(sm, A, s, a0, N);
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

__global__ void __launch_bounds__(256) k_seg_count(const int32_t* rg_off, RgView rg, int32_t* cnt) {
    const int s = blockIdx.x;
    const int r0 = rg_off[s], r1 = rg_off[s + 1];
    int c = 0;
    for (int k = r0 + threadIdx.x; k < r1; k += 256) c += is_seg(rg, r0, r1, k);
    __shared__ int tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) cnt[s] = tot;
}

__global__ void __launch_bounds__(256) k_seg_pack(const int32_t* rg_off, RgView rg, const int32_t* seg_off,
                                                  float4* geo, float* inv, uint8_t* flags) {
    const int s = blockIdx.x;
    const int r0 = rg_off[s], r1 = rg_off[s + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int wsum[8];
    int running = seg_off[s];
    for (int c0 = r0; c0 < r1; c0 += 256) {
        const int k = c0 + threadIdx.x;
        const bool f = is_seg(rg, r0, r1, k);
        const unsigned bal = __ballot_sync(kFull, f);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 8; ++w) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        if (f) {
            const int pos = running + before + __popc(bal & ((1u << lane) - 1u));
            const float ax = rg.x[k], ay = rg.y[k];
            const float ux = rg.x[k + 1] - ax, uy = rg.y[k + 1] - ay;
            geo[pos] = make_float4(ax, ay, ux, uy);
            inv[pos] = 1.0f / fmaf(ux, ux, uy * uy);
            flags[pos] = (is_seg(rg, r0, r1, k - 1) ? 1 : 0) | (is_seg(rg, r0, r1, k + 1) ? 2 : 0);
        }
        running += total;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_seg_count(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                             const uint8_t* rg_type, const uint8_t* rg_valid, int S, int32_t* cnt,
                             cudaStream_t st) {
    RgView rg{rg_x, rg_y, rg_poly, rg_type, rg_valid};
    k_seg_count<<<S, 256, 0, st>>>(rg_off, rg, cnt);
    return cudaGetLastError();
}

cudaError_t launch_seg_pack(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                            const uint8_t* rg_type, const uint8_t* rg_valid, int S, const int32_t* seg_off,
                            float4* geo, float* inv, uint8_t* flags, cudaStream_t st) {
    RgView rg{rg_x, rg_y, rg_poly, rg_type, rg_valid};
    k_seg_pack<<<S, 256, 0, st>>>(rg_off, rg, seg_off, geo, inv, flags);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t st) {
    k_step<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plain_scene(const StepArgs& a, int scene, cudaStream_t st) {
    if (a.do_transition) k_plain_transition<<<1, kThreads, 0, st>>>(a, scene);
    if (a.do_metrics) {
        k_plain_overlap<<<1, kThreads, 0, st>>>(a, scene);
        k_plain_offroad<<<1, kThreads, 0, st>>>(a, scene);
        k_plain_finish<<<1, kThreads, 0, st>>>(a, scene);
    }
    return cudaGetLastError();
}

int step_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step, kThreads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace wsim
