// Route metrics (Sec. 3.4) of each scene's first agent on its route paths:
// the route progress ratio (d_x - d_p) / (d_q - d_p) along the on-route path
// nearest to the agent, and the off-route flag (farther than route_max_dist
// from every on-route path, or nearer to an off-route path by more than
// route_max_rel).  d_x is the arc length from the path's start to the
// agent's nearest point on it; d_p, d_q those of the first and last logged
// positions.  One warp per scene: lanes take a path's segments, a
// lexicographic (distance, segment) warp minimum picks the nearest point,
// and a warp sum of the segment lengths before it gives its arc length.
#include "wsim_phases.cuh"

namespace wsim {

struct RouteArgs {
    int S, N_tot, T_log;
    const int32_t* agent_off;
    const int32_t *path_off, *path_pt_off;
    const float *path_x, *path_y;
    const uint8_t* path_on;
    const float *log_x, *log_y;
    CStateP st;
    float max_dist, max_rel;
    float* progress;
    uint8_t* off_route;
};

struct Nearest {
    float d2, arc;
    int seg;
};

// Nearest point of the polyline [k0, k1) to the point (xh + xl, yh + yl).
__device__ Nearest path_nearest(const RouteArgs& R, int k0, int k1, float xh, float xl, float yh, float yl,
                                int lane) {
    float best = WSIM_INF, bt = 0.f;
    int bs = 0x7fffffff;
    for (int k = k0 + lane; k + 1 < k1; k += 32) {
        const float ax = R.path_x[k], ay = R.path_y[k];
        const float ux = R.path_x[k + 1] - ax, uy = R.path_y[k + 1] - ay;
        const float wx = (xh - ax) + xl, wy = (yh - ay) + yl;
        const float uu = fmaf(ux, ux, uy * uy);
        const float t = uu > 0.f ? __saturatef(fmaf(wx, ux, wy * uy) / uu) : 0.f;
        const float ex = fmaf(-t, ux, wx), ey = fmaf(-t, uy, wy);
        const float d2 = fmaf(ex, ex, ey * ey);
        if (d2 < best) {  // lanes take segments in increasing order: ties keep the lower
            best = d2;
            bt = t;
            bs = k - k0;
        }
    }
    const float m = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(best)));  // d2 >= 0
    const int seg = __reduce_min_sync(kFull, static_cast<unsigned>(best == m ? bs : 0x7fffffff));
    const float t = __shfl_sync(kFull, bt, __ffs(__ballot_sync(kFull, best == m && bs == seg)) - 1);
    // arc length: the segments before `seg`, then t of segment `seg`
    float arc = 0.f, segl = 0.f;
    for (int k = k0 + lane; k + 1 < k1; k += 32) {
        const float ux = R.path_x[k + 1] - R.path_x[k], uy = R.path_y[k + 1] - R.path_y[k];
        const float l = sqrtf(fmaf(ux, ux, uy * uy));
        if (k - k0 < seg) arc += l;
        if (k - k0 == seg) segl = l;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        arc += __shfl_xor_sync(kFull, arc, o);
        segl += __shfl_xor_sync(kFull, segl, o);
    }
    return Nearest{m, fmaf(t, segl, arc), seg};
}

__global__ void __launch_bounds__(256) k_route(const RouteArgs R) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= R.S) return;
    float prog = __int_as_float(0x7fc00000);  // NaN: undefined
    uint8_t off_route = 0;
    const int g = R.agent_off[s];
    if (g < R.agent_off[s + 1]) {
        const float xh = R.st.x[g], xl = R.st.x_lo[g], yh = R.st.y[g], yl = R.st.y_lo[g];
        int best = -1;
        Nearest on{WSIM_INF, 0.f, 0};
        float off = WSIM_INF;
        for (int q = R.path_off[s]; q < R.path_off[s + 1]; ++q) {
            const Nearest h = path_nearest(R, R.path_pt_off[q], R.path_pt_off[q + 1], xh, xl, yh, yl, lane);
            if (R.path_on[q]) {
                if (h.d2 < on.d2) {
                    on = h;
                    best = q;
                }
            } else {
                off = fminf(off, h.d2);
            }
        }
        if (best >= 0) {
            const float don = sqrtf(on.d2), doff = sqrtf(off);
            off_route = don > R.max_dist || don - doff > R.max_rel;
            const int k0 = R.path_pt_off[best], k1 = R.path_pt_off[best + 1];
            const size_t last = static_cast<size_t>(R.T_log - 1) * R.N_tot + g;
            const Nearest hp = path_nearest(R, k0, k1, R.log_x[g], 0.f, R.log_y[g], 0.f, lane);
            const Nearest hq = path_nearest(R, k0, k1, R.log_x[last], 0.f, R.log_y[last], 0.f, lane);
            if (hq.arc - hp.arc > 1e-3f) prog = (on.arc - hp.arc) / (hq.arc - hp.arc);
        }
    }
    if (lane == 0) {
        R.progress[s] = prog;
        R.off_route[s] = off_route;
    }
}

cudaError_t launch_route(const StepArgs& a, const int32_t* path_off, const int32_t* path_pt_off, const float* path_x,
                         const float* path_y, const uint8_t* path_on, float max_dist, float max_rel, float* progress,
                         uint8_t* off_route, cudaStream_t st) {
    RouteArgs R{a.S, a.N_tot, a.T_log, a.agent_off, path_off, path_pt_off, path_x, path_y, path_on,
                a.log_x, a.log_y, a.in, max_dist, max_rel, progress, off_route};
    k_route<<<(a.S + 7) / 8, 256, 0, st>>>(R);
    return cudaGetLastError();
}

}  // namespace wsim
