// Observation (Sec. 3.2): for each observing agent, the other agents in its
// own frame (origin at its centre, x axis along its heading) and the K valid
// roadgraph points nearest to it (the roadgraph subsampled by distance),
// ascending, ties to the lower point index, in its frame.
//
// The ranking key of a point p is float32: c = fl(x_hi + x_lo) (the centre
// rounded once), d = fl(p - c), key = fmaf(dx, dx, dy * dy).  Rounding is
// monotone, so the same expression on a tile's bounding box clamped towards
// (or away from) c gives an exact lower (upper) bound of every key in the
// tile, with no slack.
//
// Roadgraph points are grouped in tiles of at most kPtTile consecutive
// points of one polyline (the roadgraph's own order, invalid points skipped
// in the box and the count), built once per context.  Per observer (one warp of
// k_observe_warp when K <= kObwMaxK and the observers number at least a few
// per warp that kernel keeps resident; else one CTA of k_observe):
//   1. writes the other agents in the observer's frame;
//   2. bounds the K-th key from above: a histogram of the tiles' upper bounds
//      gives a key below which whole tiles already hold K points, and a
//      histogram of the keys of the points below it tightens the bound to the
//      bucket of the K-th key;
//   3. gathers every point with key <= that bound from the tiles whose lower
//      bound is <= it (at least K points; if more than fit the shared-memory
//      list, the bound is lowered by bisection over the gathered tiles);
//   4. sorts the (key, index) pairs (bitonic, shared memory) and writes the
//      first K in the observer's frame.
#include <climits>

#include "wsim_phases.cuh"

namespace wsim {

constexpr int kObsThreads = 256;
constexpr int kObsCap = WSIM_OBS_MAX_K;  // candidate points sorted in shared memory

__device__ __forceinline__ float obs_key(float px, float py, float cx, float cy) {
    const float dx = px - cx, dy = py - cy;
    return fmaf(dx, dx, dy * dy);
}

// Tile starts of one scene.  A polyline run (consecutive points with the
// same polyline id) of L points gives ceil(L / kPtTile) tiles of consecutive
// points, so no tile spans two polylines (a tile across a gap between
// polylines has a box as large as the gap, whose lower bound then lets it
// into every nearby observer's candidates).  One CTA per scene walks its
// points in chunks: run_start(i) is the largest run start <= i (a block
// max-scan, carried across chunks), and point i starts a tile when
// i - run_start(i) is a multiple of kPtTile.  WRITE = false counts the tiles
// into out[s]; WRITE = true writes their starts to out[tile_off[s] + k] (a
// block sum-scan of the start flags) and, in the last scene, the end of the
// last tile to out[tile_off[S]].
constexpr int kPtThreads = 1024;

template <bool MAX>
__device__ __forceinline__ int block_scan(int v, int* wtot) {  // inclusive, kPtThreads threads
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = MAX ? max(v, u) : v + u;
    }
    if (lane == 31) wtot[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = wtot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x = MAX ? max(x, u) : x + u;
        }
        wtot[lane] = x;
    }
    __syncthreads();
    const int before = w > 0 ? wtot[w - 1] : (MAX ? -1 : 0);
    return MAX ? max(v, before) : v + before;
}

template <bool WRITE>
__global__ void __launch_bounds__(kPtThreads) k_pt_starts(const int32_t* rg_off, const int32_t* rg_poly,
                                                          const int32_t* tile_off, int S, int32_t* out) {
    __shared__ int wmax[32], wsum[32];
    __shared__ int carry_rs, carry_n;
    const int s = blockIdx.x;
    const int r0 = rg_off[s], r1 = rg_off[s + 1];
    if (threadIdx.x == 0) {
        carry_rs = r0;
        carry_n = 0;
    }
    __syncthreads();
    for (int base = r0; base < r1; base += kPtThreads) {
        const int i = base + threadIdx.x;
        const bool in = i < r1;
        const bool rs = in && (i == r0 || rg_poly[i] != rg_poly[i - 1]);
        const int run_start = max(carry_rs, block_scan<true>(rs ? i : -1, wmax));
        const int st = in && (i - run_start) % kPtTile == 0;
        const int incl = block_scan<false>(st, wsum) + carry_n;
        if (WRITE && st) out[tile_off[s] + incl - 1] = i;
        __syncthreads();  // every thread has read the carries
        if (threadIdx.x == kPtThreads - 1) {
            carry_rs = run_start;
            carry_n = incl;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (!WRITE) out[s] = carry_n;
        if (WRITE && s == S - 1) out[tile_off[S]] = r1;
    }
}

// Tile boxes: (xmin, ymin, xmax, ymax) of the valid points and their count.
__global__ void __launch_bounds__(256) k_pt_tiles(const int32_t* tile_off, const int32_t* pt_start, const float* rg_x,
                                                  const float* rg_y, const uint8_t* rg_valid, int S, float4* box,
                                                  int32_t* cnt) {
    const int s = blockIdx.x;
    const int t0 = tile_off[s], nt = tile_off[s + 1] - t0;
    for (int t = threadIdx.x; t < nt; t += 256) {
        float x0 = WSIM_INF, y0 = WSIM_INF, x1 = -WSIM_INF, y1 = -WSIM_INF;
        int n = 0;
        const int a = pt_start[t0 + t], b = pt_start[t0 + t + 1];
        for (int r = a; r < b; ++r) {
            if (!rg_valid[r]) continue;
            const float x = rg_x[r], y = rg_y[r];
            x0 = fminf(x0, x);
            x1 = fmaxf(x1, x);
            y0 = fminf(y0, y);
            y1 = fmaxf(y1, y);
            ++n;
        }
        box[t0 + t] = make_float4(x0, y0, x1, y1);
        cnt[t0 + t] = n;
    }
}

// Observers in a list, ascending within each warp's 32 agents (consecutive
// entries mostly share a scene and its roadgraph in L1).
__global__ void k_obs_list(const uint8_t* observers, const uint8_t* valid, int N_tot, int32_t* list, int32_t* count) {
    for (int base = blockIdx.x * blockDim.x; base < N_tot; base += gridDim.x * blockDim.x) {
        const int g = base + threadIdx.x, lane = threadIdx.x & 31;
        const bool obs = g < N_tot && (observers ? observers[g] != 0 : valid[g] != 0);
        const unsigned bal = __ballot_sync(0xffffffffu, obs);
        int pos = 0;
        if (lane == 0 && bal) pos = atomicAdd(count, __popc(bal));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (obs) list[pos + __popc(bal & ((1u << lane) - 1u))] = g;
    }
}

// Key histogram: the top 10 bits of the float (half an octave per bucket);
// 12 bits (an eighth of an octave) took 16 % longer on all-agent observation
// (clearing and scanning the bins), 9 and 8 bits gather too many points.
constexpr int kHistBits = 10;
constexpr int kObsTiles = 1500;  // tiles whose upper bound and count are cached per observer
constexpr int kObsList = 1000;   // tiles that can hold a point below the bound (48 KB static in all)

struct ObsSmem {
    unsigned long long item[kObsCap];  // (key bits << 32) | point index
    float tmax[kObsTiles];             // per tile: upper bound of its keys (+inf: empty)
    int tcnt[kObsTiles];
    int list[kObsList];                // tiles whose lower bound is <= the tile bound
    int red[kObsThreads / 32];
    int n, nlist;
};

__device__ __forceinline__ int block_sum(int v, ObsSmem& sm) {
    v = __reduce_add_sync(kFull, v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm.red[w] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int k = 0; k < kObsThreads / 32; ++k) t += sm.red[k];
    return t;
}

// Upper bound of the keys of tile B (the box corner farthest from c).
__device__ __forceinline__ float tile_upper(const float4 B, float cx, float cy) {
    const float fx = fmaxf(fabsf(B.x - cx), fabsf(B.z - cx)), fy = fmaxf(fabsf(B.y - cy), fabsf(B.w - cy));
    return fmaf(fx, fx, fy * fy);
}

// Lower bound of the keys of tile B (the box clamped towards c).
__device__ __forceinline__ float tile_lower(const float4 B, float cx, float cy) {
    const float nx = fminf(fmaxf(cx, B.x), B.z), ny = fminf(fmaxf(cy, B.y), B.w);
    return obs_key(nx, ny, cx, cy);
}

// The first bucket of hist (1 << kHistBits counts) at which the running
// total reaches `want` (-1 if it never does); *upto = the total up to and
// including that bucket.  Block-wide, ends with a barrier.
__device__ int hist_crossing(const int* hist, int want, ObsSmem& sm, int* upto) {
    constexpr int H = 1 << kHistBits, per = H / kObsThreads;
    int local = 0;
    for (int k = 0; k < per; ++k) local += hist[threadIdx.x * per + k];
    int incl = local;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) sm.red[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += sm.red[w];
    incl += before;
    const int excl = incl - local;
    __shared__ int found[2];
    if (threadIdx.x == 0) found[0] = -1;
    __syncthreads();
    if (excl < want && incl >= want) {  // the crossing bucket is in this thread's range
        int run = excl, b = threadIdx.x * per;
        while (run + hist[b] < want) run += hist[b++];
        found[0] = b;
        found[1] = run + hist[b];
    }
    __syncthreads();
    const int b = found[0];
    *upto = b >= 0 ? found[1] : 0;
    __syncthreads();
    return b;
}

// A tighter bound from the points themselves: a histogram of the keys of
// every point in the tiles that can hold one below tau gives the top of the
// bucket holding the want-th key; *n = the points at or below it.
__device__ float point_bound(const float4* box, const int32_t* cnt, int t0, int nt, const int32_t* ps, const float* rg_x,
                             const float* rg_y, const uint8_t* rg_valid, float cx, float cy, float tau, int want,
                             ObsSmem& sm, int* n) {
    int* hist = reinterpret_cast<int*>(sm.item);
    constexpr int H = 1 << kHistBits;
    for (int i = threadIdx.x; i < H; i += kObsThreads) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nl = sm.nlist, m = nl >= 0 ? nl : nt;
    for (int q = warp; q < m; q += kObsThreads / 32) {
        const int t = nl >= 0 ? sm.list[q] : q;
        if (nl < 0 && (cnt[t0 + t] == 0 || tile_lower(box[t0 + t], cx, cy) > tau)) continue;
        const int r = ps[t] + lane;
        if (r < ps[t + 1] && rg_valid[r]) {
            const float key = obs_key(rg_x[r], rg_y[r], cx, cy);
            if (key <= tau && key < WSIM_INF) atomicAdd(&hist[__float_as_uint(key) >> (32 - kHistBits)], 1);
        }
    }
    __syncthreads();
    const int b = hist_crossing(hist, want, sm, n);
    if (b < 0) {  // fewer finite keys than wanted below tau: keep tau
        *n = -1;
        return tau;
    }
    return fminf(tau, __uint_as_float(((static_cast<uint32_t>(b) + 1u) << (32 - kHistBits)) - 1u));
}

// An upper bound tau of the want-th smallest key: the tiles' upper bounds
// are counted in a histogram of their float bits' top kHistBits bits (keys
// are >= 0, so bits order like values; a bucket spans half an octave), and tau
// is the top of the first bucket at which the counts reach `want`: every tile
// up to that bucket lies entirely within tau.  Tiles whose bounds overflow
// (+inf) never count; if they would be needed, tau = +inf.

__device__ float tile_bound(const float4* box, const int32_t* cnt, int t0, int nt, float cx, float cy, int want,
                            ObsSmem& sm) {
    int* hist = reinterpret_cast<int*>(sm.item);  // the item list is free until the gather
    constexpr int H = 1 << kHistBits;
    for (int i = threadIdx.x; i < H; i += kObsThreads) hist[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += kObsThreads) {
        float u;
        int n;
        if (t < kObsTiles) {
            u = sm.tmax[t];
            n = sm.tcnt[t];
        } else {
            n = cnt[t0 + t];
            u = n > 0 ? tile_upper(box[t0 + t], cx, cy) : WSIM_INF;
        }
        if (n > 0 && u < WSIM_INF) atomicAdd(&hist[__float_as_uint(u) >> (32 - kHistBits)], n);
    }
    __syncthreads();
    int total;
    const int b = hist_crossing(hist, want, sm, &total);
    if (b < 0) return WSIM_INF;
    return __uint_as_float(((static_cast<uint32_t>(b) + 1u) << (32 - kHistBits)) - 1u);
}


// Points with key <= tau in the tiles that can hold one.
__device__ int count_points_within(const float4* box, const int32_t* cnt, int t0, int nt, const int32_t* ps,
                                   const float* rg_x, const float* rg_y, const uint8_t* rg_valid, float cx, float cy,
                                   float tau, ObsSmem& sm) {
    int c = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nl = sm.nlist, m = nl >= 0 ? nl : nt;
    for (int q = warp; q < m; q += kObsThreads / 32) {
        const int t = nl >= 0 ? sm.list[q] : q;
        if (nl < 0 && (cnt[t0 + t] == 0 || tile_lower(box[t0 + t], cx, cy) > tau)) continue;
        const int r = ps[t] + lane;
        if (r < ps[t + 1] && rg_valid[r] && obs_key(rg_x[r], rg_y[r], cx, cy) <= tau) ++c;
    }
    return block_sum(c, sm);
}

// The other agents of the observer's scene in its frame (position, heading
// difference, velocity); slots j >= N, the observer itself and invalid agents
// are zero and flagged invalid.  Threads j0, j0 + stride, ... of the caller.
__device__ __forceinline__ void agents_in_frame(const StepArgs& A, int g, int a0, int N, int M, float xh, float xl,
                                                float yh, float yl, float th, float tl, float c, float sn, int j0,
                                                int stride, float* agents, uint8_t* agents_valid) {
    for (int j = j0; j < M; j += stride) {
        const int gj = a0 + j;
        const bool ok = j < N && gj != g && A.valid[gj];
        const size_t o = static_cast<size_t>(g) * M + j;
        float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
            const float dx = comp_diff(A.in.x[gj], A.in.x_lo[gj], xh, xl);
            const float dy = comp_diff(A.in.y[gj], A.in.y_lo[gj], yh, yl);
            v[0] = fmaf(c, dx, sn * dy);
            v[1] = fmaf(-sn, dx, c * dy);
            v[2] = turn_from(A.in.th[gj], th, tl - A.in.th_lo[gj]);  // heading difference mod 2 pi
            const float vx = A.in.vx[gj], vy = A.in.vy[gj];
            v[3] = fmaf(c, vx, sn * vy);
            v[4] = fmaf(-sn, vx, c * vy);
        }
        agents_valid[o] = ok;
#pragma unroll
        for (int k = 0; k < 5; ++k) agents[o * 5 + k] = v[k];
    }
}

// The first `have` sorted items as the observer's K points in its frame;
// slots k >= have get index -1.  Threads k0, k0 + stride, ... of the caller.
__device__ __forceinline__ void write_points(const unsigned long long* item, int g, int K, int have, const float* rg_x,
                                             const float* rg_y, float xh, float xl, float yh, float yl, float c,
                                             float sn, int k0, int stride, float* rg_out, int32_t* rg_idx) {
    for (int k = k0; k < K; k += stride) {
        const size_t o = static_cast<size_t>(g) * K + k;
        float ox = 0.f, oy = 0.f;
        int idx = -1;
        if (k < have) {
            idx = static_cast<int>(item[k] & 0xffffffffull);
            const float dx = comp_diff(rg_x[idx], 0.f, xh, xl);
            const float dy = comp_diff(rg_y[idx], 0.f, yh, yl);
            ox = fmaf(c, dx, sn * dy);
            oy = fmaf(-sn, dx, c * dy);
        }
        rg_out[2 * o] = ox;
        rg_out[2 * o + 1] = oy;
        rg_idx[o] = idx;
    }
}

__global__ void __launch_bounds__(kObsThreads) k_observe(const StepArgs A, const int32_t* list, const int32_t* count,
                                                         const float* rg_x, const float* rg_y,
                                                         const uint8_t* rg_valid, const int32_t* tile_off,
                                                         const int32_t* pt_start, const float4* box,
                                                         const int32_t* cnt, int M, int K,
                                                         float* agents, uint8_t* agents_valid, float* rg_out,
                                                         int32_t* rg_idx, const int32_t* scene_of, int N_tot,
                                                         int warp_min) {
    __shared__ ObsSmem sm;
    // Below warp_min observers this kernel observes them all; else only the
    // warp kernel's overflow list (list + N_tot, count[2]).
    const bool all = count[0] < warp_min;
    const int n_obs = all ? count[0] : count[2];
    const int32_t* obs_list = all ? list : list + N_tot;
    for (int q = blockIdx.x; q < n_obs; q += gridDim.x) {
        const int g = obs_list[q];
        const int s = scene_of[g];
        const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
        const float xh = A.in.x[g], xl = A.in.x_lo[g], yh = A.in.y[g], yl = A.in.y_lo[g];
        const float th = A.in.th[g], tl = A.in.th_lo[g];
        float c, sn;
        comp_sincos(th, tl, c, sn);
        // 1. Other agents in the observer's frame.
        agents_in_frame(A, g, a0, N, M, xh, xl, yh, yl, th, tl, c, sn, threadIdx.x, kObsThreads, agents, agents_valid);
        // 2. Upper bound of the K-th key from the tiles.
        const int t0 = tile_off[s], nt = tile_off[s + 1] - t0;
        const int32_t* ps = pt_start + t0;  // tile t: points ps[t] .. ps[t+1]-1
        const float cx = __fadd_rn(xh, xl), cy = __fadd_rn(yh, yl);
        int total = 0;
        for (int t = threadIdx.x; t < nt; t += kObsThreads) {
            const int n = cnt[t0 + t];
            total += n;
            if (t < kObsTiles) {
                sm.tcnt[t] = n;
                sm.tmax[t] = n > 0 ? tile_upper(box[t0 + t], cx, cy) : WSIM_INF;
            }
        }
        total = block_sum(total, sm);  // its barriers also publish the cache
        const int want = min(K, total);
        float tau = WSIM_INF;
        if (want > 0) tau = tile_bound(box, cnt, t0, nt, cx, cy, want, sm);
        // the tiles that can hold a point below tau (-1: more than fit, scan all)
        if (threadIdx.x == 0) sm.nlist = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += kObsThreads) {
            const bool in = cnt[t0 + t] > 0 && tile_lower(box[t0 + t], cx, cy) <= tau;
            if (in) {
                const int q = atomicAdd(&sm.nlist, 1);
                if (q < kObsList) sm.list[q] = t;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && sm.nlist > kObsList) sm.nlist = -1;
        __syncthreads();
        // 3. Gather (lowering tau while the list would overflow).
        int n = 0;
        if (want > 0) {
            tau = point_bound(box, cnt, t0, nt, ps, rg_x, rg_y, rg_valid, cx, cy, tau, want, sm, &n);
            if (n < 0) n = count_points_within(box, cnt, t0, nt, ps, rg_x, rg_y, rg_valid, cx, cy, tau, sm);
        }
        if (n > kObsCap) {
            uint32_t lo = 0, hi = __float_as_uint(tau);
            while (lo < hi) {  // smallest tau' with at least `want` points
                const uint32_t mid = lo + (hi - lo) / 2;
                if (count_points_within(box, cnt, t0, nt, ps, rg_x, rg_y, rg_valid, cx, cy, __uint_as_float(mid),
                                        sm) >= want)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            tau = __uint_as_float(lo);
            n = count_points_within(box, cnt, t0, nt, ps, rg_x, rg_y, rg_valid, cx, cy, tau, sm);
            if (n > kObsCap) {  // more than kObsCap points share the K-th key
                if (threadIdx.x == 0) set_status(A.status, WSIM_ESIZE);
                n = 0;
            }
        }
        if (threadIdx.x == 0) sm.n = 0;
        __syncthreads();
        if (n > 0) {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const int nl = sm.nlist, m = nl >= 0 ? nl : nt;
            for (int qq = warp; qq < m; qq += kObsThreads / 32) {
                const int t = nl >= 0 ? sm.list[qq] : qq;
                if (nl < 0 && (cnt[t0 + t] == 0 || tile_lower(box[t0 + t], cx, cy) > tau)) continue;
                const int r = ps[t] + lane;
                float key = 0.f;
                const bool in = r < ps[t + 1] && rg_valid[r] && (key = obs_key(rg_x[r], rg_y[r], cx, cy)) <= tau;
                const unsigned bal = __ballot_sync(kFull, in);
                int base = 0;
                if (lane == 0 && bal) base = atomicAdd(&sm.n, __popc(bal));
                base = __shfl_sync(kFull, base, 0);
                if (in)
                    sm.item[base + __popc(bal & ((1u << lane) - 1u))] =
                        (static_cast<unsigned long long>(__float_as_uint(key)) << 32) | static_cast<uint32_t>(r);
            }
        }
        __syncthreads();
        // 4. Bitonic sort of the gathered items (padded to a power of two).
        int p2 = 1;
        while (p2 < n) p2 <<= 1;
        for (int i = n + threadIdx.x; i < p2; i += kObsThreads) sm.item[i] = ~0ull;
        __syncthreads();
        for (int size = 2; size <= p2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < p2 / 2; i += kObsThreads) {
                    const int lo = 2 * i - (i & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long a = sm.item[lo], b = sm.item[hi];
                    if ((a > b) == up) {
                        sm.item[lo] = b;
                        sm.item[hi] = a;
                    }
                }
                __syncthreads();
            }
        }
        write_points(sm.item, g, K, min(want, n), rg_x, rg_y, xh, xl, yh, yl, c, sn, threadIdx.x, kObsThreads, rg_out,
                     rg_idx);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp per observer (K <= kObwMaxK, at least one observer per resident
// warp): the same four steps with a histogram, tile list
// and point list private to each warp, so that no step waits at a block
// barrier.  Warps take chunks of kObwChunk consecutive list entries from a
// counter.  An observer whose gathered points would exceed kObwCap goes to the
// block kernel's overflow list instead, which then observes it from the start.
// The tile and point passes take four tiles per iteration (their loads in
// flight together: one warp's chain of dependent loads is the cost).
constexpr int kObwWarps = 8;
constexpr int kObwCap = 512;    // gathered points per warp
constexpr int kObwList = 128;   // candidate tiles per warp (more: every tile is re-tested)
constexpr int kObwChunk = 1;   // observers taken from the counter at a time (larger chunks left a longer tail)
constexpr int kObwMaxK = kObwCap / 2;
constexpr int kObwU = 4;         // tiles whose loads a pass issues together
static_assert(kObwCap * 2 >= (1 << kHistBits), "the key histogram shares the point list");

struct ObwSmem {
    unsigned long long item[kObwWarps][kObwCap];
    int start[kObwWarps][kObwList];      // candidate tiles: first point,
    float lower[kObwWarps][kObwList];    // ... lower bound of their keys
    uint8_t len[kObwWarps][kObwList];    // ... and point count (<= kPtTile)
};

// The top of key-histogram bucket b (the largest float bit pattern in it).
__device__ __forceinline__ float bucket_top(int b) {
    return __uint_as_float(((static_cast<uint32_t>(b) + 1u) << (32 - kHistBits)) - 1u);
}

__device__ __forceinline__ void warp_clear_hist(int* hist, int lane) {
    int4* h4 = reinterpret_cast<int4*>(hist);
#pragma unroll
    for (int i = 0; i < (1 << kHistBits) / 128; ++i) h4[i * 32 + lane] = make_int4(0, 0, 0, 0);
    __syncwarp();
}

// The first bucket of hist at which the running total reaches want > 0 (-1
// if it never does); *upto = the total through that bucket.
__device__ __forceinline__ int warp_crossing(const int* hist, int want, int lane, int* upto) {
    constexpr int per = (1 << kHistBits) / 32;
    const int4* h4 = reinterpret_cast<const int4*>(hist + lane * per);
    int local = 0;
#pragma unroll
    for (int k = 0; k < per / 4; ++k) {
        const int4 v = h4[k];
        local += (v.x + v.y) + (v.z + v.w);
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned hit = __ballot_sync(kFull, incl >= want);
    if (!hit) {
        *upto = 0;
        return -1;
    }
    const int src = __ffs(hit) - 1;
    int b = 0, run = 0;
    if (lane == src) {
        run = incl - local;
        b = lane * per;
        while (run + hist[b] < want) run += hist[b++];
        run += hist[b];
    }
    *upto = __shfl_sync(kFull, run, src);
    return __shfl_sync(kFull, b, src);
}

// Visits the points of the candidate tiles (nl >= 0: the nl listed ones,
// tile q's points ts[q] .. ts[q] + tn[q] - 1, four tiles' loads in flight at
// a time; else every tile whose box can hold a point with key <= tau, tile
// t's points ps[t] .. ps[t+1]-1): f(ok, key, r) on every lane for every
// tile, ok = the lane's point exists and is valid (warp-uniform calls: f may
// use warp votes).
template <class F>
__device__ __forceinline__ void warp_points(const int* ts, const uint8_t* tn, int nl, int nt, const float4* box,
                                            const int32_t* cnt, int t0, const int32_t* ps, const float* rg_x,
                                            const float* rg_y, const uint8_t* rg_valid, float cx, float cy, float tau,
                                            int lane, F f) {
    if (nl >= 0) {
        for (int q = 0; q < nl; q += kObwU) {
            float x[kObwU], y[kObwU];
            bool ok[kObwU];
            int r[kObwU];
#pragma unroll
            for (int u = 0; u < kObwU; ++u) {
                const bool has = q + u < nl;
                r[u] = (has ? ts[q + u] : ts[0]) + lane;
                const bool in = has && lane < tn[q + u];
                const int rr = in ? r[u] : ts[0];  // a listed tile's first point (nl > 0 here)
                x[u] = rg_x[rr];
                y[u] = rg_y[rr];
                const uint8_t v = rg_valid[rr];
                ok[u] = in && v;
            }
#pragma unroll
            for (int u = 0; u < kObwU; ++u) f(ok[u], obs_key(x[u], y[u], cx, cy), r[u]);
        }
    } else {
        for (int t = 0; t < nt; ++t) {
            if (cnt[t0 + t] == 0 || tile_lower(box[t0 + t], cx, cy) > tau) continue;
            const int r = ps[t] + lane;
            const bool ok = r < ps[t + 1] && rg_valid[r];
            f(ok, ok ? obs_key(rg_x[r], rg_y[r], cx, cy) : 0.f, r);
        }
    }
}

// One compare-exchange stage of the bitonic network over item[0, p2) (the
// rule of the block kernel's sort: pair (lo, lo + stride), ascending where
// lo & size is 0).
__device__ __forceinline__ void bitonic_stage(unsigned long long* item, int p2, int size, int stride, int lane) {
    for (int i = lane; i < p2 / 2; i += 32) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = item[lo], b = item[hi];
        if ((a > b) == up) {
            item[lo] = b;
            item[hi] = a;
        }
    }
    __syncwarp();
}

// The stages of strides below kSortChunk act within aligned chunks of
// kSortChunk items, so a lane runs them on a chunk held in registers: the
// chunk sort (sizes 2 .. kSortChunk) and, after each larger size's
// shared-memory stages, its last three strides.  28 shared-memory round
// trips instead of 45 for 512 items; the same network, so the same order.
constexpr int kSortChunk = 8;
__device__ __forceinline__ void cswap(unsigned long long& a, unsigned long long& b, bool up) {
    const unsigned long long x = a, y = b;
    const bool sw = (x > y) == up;
    a = sw ? y : x;
    b = sw ? x : y;
}

// Sorts item[0, p2) ascending (p2 a power of two, <= kObwCap), warp-wide.
__device__ void warp_bitonic(unsigned long long* item, int p2, int lane) {
    if (p2 < kSortChunk) {
        for (int size = 2; size <= p2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) bitonic_stage(item, p2, size, stride, lane);
        return;
    }
    const int nc = p2 / kSortChunk;
    for (int ch = lane; ch < nc; ch += 32) {  // chunk sort, directions of the whole network
        unsigned long long v[kSortChunk];
        const int base = ch * kSortChunk;
#pragma unroll
        for (int k = 0; k < kSortChunk; ++k) v[k] = item[base + k];
#pragma unroll
        for (int size = 2; size <= kSortChunk; size <<= 1)
#pragma unroll
            for (int st = size >> 1; st > 0; st >>= 1)
#pragma unroll
                for (int k = 0; k < kSortChunk; ++k)
                    if (!(k & st)) cswap(v[k], v[k + st], ((base + k) & size) == 0);
#pragma unroll
        for (int k = 0; k < kSortChunk; ++k) item[base + k] = v[k];
    }
    __syncwarp();
    for (int size = 2 * kSortChunk; size <= p2; size <<= 1) {
        for (int stride = size >> 1; stride >= kSortChunk; stride >>= 1) bitonic_stage(item, p2, size, stride, lane);
        for (int ch = lane; ch < nc; ch += 32) {  // strides 4, 2, 1: one direction per chunk
            unsigned long long v[kSortChunk];
            const int base = ch * kSortChunk;
            const bool up = (base & size) == 0;
#pragma unroll
            for (int k = 0; k < kSortChunk; ++k) v[k] = item[base + k];
#pragma unroll
            for (int st = kSortChunk / 2; st > 0; st >>= 1)
#pragma unroll
                for (int k = 0; k < kSortChunk; ++k)
                    if (!(k & st)) cswap(v[k], v[k + st], up);
#pragma unroll
            for (int k = 0; k < kSortChunk; ++k) item[base + k] = v[k];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kObwWarps * 32, 5)
    k_observe_warp(const StepArgs A, const int32_t* list, int32_t* count, int warp_min,
                   const float* rg_x, const float* rg_y, const uint8_t* rg_valid, const int32_t* tile_off,
                   const int32_t* pt_start,
                   const float4* box, const int32_t* cnt, int M, int K, float* agents, uint8_t* agents_valid,
                   float* rg_out, int32_t* rg_idx, const int32_t* scene_of) {
    static_assert(kPtTile == 32, "a tile's points are the warp's lanes");
    __shared__ ObwSmem sm;
    const int n_obs = count[0];
    if (n_obs < warp_min) return;  // the block kernel observes them all
    int32_t* ovf_list = const_cast<int32_t*>(list) + A.N_tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* item = sm.item[w];
    int* hist = reinterpret_cast<int*>(item);  // free until the gather
    int* ts = sm.start[w];
    float* tlb = sm.lower[w];
    uint8_t* tn = sm.len[w];
    const unsigned below = (1u << lane) - 1u;
    const int nchunks = (n_obs + kObwChunk - 1) / kObwChunk;
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(count + 1, 1);
        ch = __shfl_sync(kFull, ch, 0);
        if (ch >= nchunks) break;
        const int e0 = ch * kObwChunk, e1 = min(n_obs, e0 + kObwChunk);
        for (int e = e0; e < e1; ++e) {
            const int g = list[e];
            const int s = scene_of[g];
            const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
            const float xh = A.in.x[g], xl = A.in.x_lo[g], yh = A.in.y[g], yl = A.in.y_lo[g];
            const float th = A.in.th[g], tlo = A.in.th_lo[g];
            float c, sn;
            comp_sincos(th, tlo, c, sn);
            // 1. Other agents in the observer's frame.
            agents_in_frame(A, g, a0, N, M, xh, xl, yh, yl, th, tlo, c, sn, lane, 32, agents, agents_valid);
            // 2. Upper bound of the K-th key from the tiles, and the valid-point total.
            const int t0 = tile_off[s], nt = tile_off[s + 1] - t0;
            const int32_t* ps = pt_start + t0;  // tile t: points ps[t] .. ps[t+1]-1
            const float cx = __fadd_rn(xh, xl), cy = __fadd_rn(yh, yl);
            warp_clear_hist(hist, lane);
            int total = 0;
            for (int tb = 0; tb < nt; tb += kObwU * 32) {
                int n[kObwU];
                float4 B[kObwU];
#pragma unroll
                for (int u = 0; u < kObwU; ++u) {
                    const int t = min(tb + 32 * u + lane, nt - 1);
                    n[u] = cnt[t0 + t];
                    B[u] = box[t0 + t];
                }
#pragma unroll
                for (int u = 0; u < kObwU; ++u) {
                    if (tb + 32 * u + lane >= nt) n[u] = 0;
                    total += n[u];
                    if (n[u] > 0) {
                        const float up = tile_upper(B[u], cx, cy);
                        if (up < WSIM_INF) atomicAdd(&hist[__float_as_uint(up) >> (32 - kHistBits)], n[u]);
                    }
                }
            }
            total = __reduce_add_sync(kFull, total);
            __syncwarp();
            const int want = min(K, total);
            int n = 0;
            if (want > 0) {
                int upto;
                const int b = warp_crossing(hist, want, lane, &upto);
                float tau = b < 0 ? WSIM_INF : bucket_top(b);
                // 3. The tiles that can hold a point below tau (nl = -1: more than fit).
                int nl = 0;
                for (int tb = 0; tb < nt; tb += kObwU * 32) {
                    bool in[kObwU];
                    float lo[kObwU];
#pragma unroll
                    for (int u = 0; u < kObwU; ++u) {
                        const int t = min(tb + 32 * u + lane, nt - 1);
                        const int c1 = cnt[t0 + t];
                        const float4 B = box[t0 + t];
                        lo[u] = tile_lower(B, cx, cy);
                        in[u] = tb + 32 * u + lane < nt && c1 > 0 && lo[u] <= tau;
                    }
#pragma unroll
                    for (int u = 0; u < kObwU; ++u) {
                        const unsigned bal = __ballot_sync(kFull, in[u]);
                        const int q = nl + __popc(bal & below);
                        if (in[u] && q < kObwList) {
                            const int t = tb + 32 * u + lane;
                            ts[q] = ps[t];
                            tn[q] = static_cast<uint8_t>(ps[t + 1] - ps[t]);
                            tlb[q] = lo[u];
                        }
                        nl += __popc(bal);
                    }
                }
                if (nl > kObwList) nl = -1;
                __syncwarp();
                // 4. A histogram of the candidate points' keys tightens tau.
                warp_clear_hist(hist, lane);
                warp_points(ts, tn, nl, nt, box, cnt, t0, ps, rg_x, rg_y, rg_valid, cx, cy, tau, lane,
                            [&](bool ok, float key, int) {
                                if (ok && key <= tau && key < WSIM_INF)
                                    atomicAdd(&hist[__float_as_uint(key) >> (32 - kHistBits)], 1);
                            });
                __syncwarp();
                const int b2 = warp_crossing(hist, want, lane, &n);
                __syncwarp();  // the histogram is read before the gather overwrites it
                if (b2 >= 0) {
                    tau = fminf(tau, bucket_top(b2));
                    // keep the listed tiles that can still hold a point below the
                    // tightened tau (in place: a round reads before it writes)
                    if (nl > 0) {
                        int nk = 0;
                        for (int qb = 0; qb < nl; qb += 32) {
                            const int qq = qb + lane;
                            const bool keep = qq < nl && tlb[qq] <= tau;
                            const int a1 = keep ? ts[qq] : 0;
                            const float l1 = keep ? tlb[qq] : 0.f;
                            const uint8_t n1 = keep ? tn[qq] : 0;
                            const unsigned bal = __ballot_sync(kFull, keep);
                            const int d = nk + __popc(bal & below);
                            __syncwarp();  // the round's entries are read before any is overwritten
                            if (keep) {
                                ts[d] = a1;
                                tlb[d] = l1;
                                tn[d] = n1;
                            }
                            nk += __popc(bal);
                            __syncwarp();
                        }
                        nl = nk;
                    }
                } else {  // fewer finite keys than wanted below tau: keep tau
                    int c1 = 0;
                    warp_points(ts, tn, nl, nt, box, cnt, t0, ps, rg_x, rg_y, rg_valid, cx, cy, tau, lane,
                                [&](bool ok, float key, int) { c1 += ok && key <= tau; });
                    n = __reduce_add_sync(kFull, c1);
                }
                if (n > kObwCap) {  // the block kernel observes this one
                    if (lane == 0) ovf_list[atomicAdd(count + 2, 1)] = g;
                    continue;
                }
                // 5. Gather the points with key <= tau (exactly n of them).
                int base = 0;
                warp_points(ts, tn, nl, nt, box, cnt, t0, ps, rg_x, rg_y, rg_valid, cx, cy, tau, lane,
                            [&](bool ok, float key, int r) {
                                const bool in = ok && key <= tau;
                                const unsigned bal = __ballot_sync(kFull, in);
                                const int pos = base + __popc(bal & below);
                                if (in && pos < kObwCap)
                                    item[pos] = (static_cast<unsigned long long>(__float_as_uint(key)) << 32) |
                                                static_cast<uint32_t>(r);
                                base += __popc(bal);
                            });
                n = min(base, kObwCap);
                // 6. Bitonic sort of (key, index), padded to a power of two.
                int p2 = 1;
                while (p2 < n) p2 <<= 1;
                for (int i = n + lane; i < p2; i += 32) item[i] = ~0ull;
                __syncwarp();
                warp_bitonic(item, p2, lane);
            }
            // 7. The first K in the observer's frame.
            write_points(item, g, K, min(want, n), rg_x, rg_y, xh, xl, yh, yl, c, sn, lane, 32, rg_out, rg_idx);
            __syncwarp();
        }
    }
}

cudaError_t launch_pt_count(const int32_t* rg_off, const int32_t* rg_poly, int S, int32_t* tiles_per_scene,
                            cudaStream_t st) {
    k_pt_starts<false><<<S, kPtThreads, 0, st>>>(rg_off, rg_poly, nullptr, S, tiles_per_scene);
    return cudaGetLastError();
}

cudaError_t launch_pt_tiles(const int32_t* rg_off, const int32_t* rg_poly, const int32_t* tile_off, const float* rg_x,
                            const float* rg_y, const uint8_t* rg_valid, int S, int32_t* pt_start, float4* box,
                            int32_t* cnt, cudaStream_t st) {
    k_pt_starts<true><<<S, kPtThreads, 0, st>>>(rg_off, rg_poly, tile_off, S, pt_start);
    k_pt_tiles<<<S, 256, 0, st>>>(tile_off, pt_start, rg_x, rg_y, rg_valid, S, box, cnt);
    return cudaGetLastError();
}

cudaError_t launch_observe(const StepArgs& a, const uint8_t* observers, int32_t* list, int32_t* count,
                           const float* rg_x, const float* rg_y, const uint8_t* rg_valid, const int32_t* tile_off,
                           const int32_t* pt_start, const float4* box, const int32_t* cnt, const int32_t* scene_of,
                           int M, int K, float* agents, uint8_t* agents_valid, float* rg, int32_t* rg_idx,
                           cudaStream_t st) {
    // list[0, N): the observers, count[0] of them; count[1]: the warp kernel's
    // chunk counter; list[N, 2N) and count[2]: its overflow to the block kernel.
    cudaError_t e = cudaMemsetAsync(count, 0, 3 * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (a.N_tot == 0) return cudaSuccess;
    int dev = 0, sms = 148, per = 1, perw = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = std::min((a.N_tot + 255) / 256, 4096);
    k_obs_list<<<std::max(nb, 1), 256, 0, st>>>(observers, a.valid, a.N_tot, list, count);
    // The warp kernel takes over from one observer per resident warp: each
    // warp's observer is a serial chain, so with fewer observers than warps
    // the block kernel's finer grain wins (30k-point scenes, K = 256: 2,048
    // observers 0.15 ms on the block kernel against 0.18 on the warp kernel;
    // 16,384 observers 0.77 against 0.49 ms).
    int warp_min = INT_MAX;
    if (K <= kObwMaxK) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perw, k_observe_warp, kObwWarps * 32, 0);
        warp_min = sms * std::max(perw, 1) * kObwWarps;
        k_observe_warp<<<sms * std::max(perw, 1), kObwWarps * 32, 0, st>>>(
            a, list, count, warp_min, rg_x, rg_y, rg_valid, tile_off, pt_start, box, cnt, M, K, agents,
            agents_valid, rg, rg_idx, scene_of);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_observe, kObsThreads, 0);
    k_observe<<<sms * std::max(per, 1), kObsThreads, 0, st>>>(a, list, count, rg_x, rg_y, rg_valid, tile_off,
                                                              pt_start, box, cnt, M, K, agents, agents_valid, rg,
                                                              rg_idx, scene_of, a.N_tot, warp_min);
    return cudaGetLastError();
}

}  // namespace wsim
