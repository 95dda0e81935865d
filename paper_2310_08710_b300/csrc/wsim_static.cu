// wsim_metrics_static: the metrics pass (overlap, off-road, log divergence,
// reward) for callers that may not allocate device memory.
//
// Some hosts cannot call cudaMalloc at the point where they need the
// metrics: an allocator that owns every byte of the device (a framework's
// caching pool, a fixed arena of an embedded or real-time system), or code
// running where allocation is forbidden.  This entry point keeps the scratch
// that wsim_init would allocate (packed road-edge segments, per-scene
// offsets, work counter, status word) in one file-scope device array of fixed
// size instead, and allocates nothing.  The caller still passes the scene
// batch, the state and the metric arrays.
#include <cstring>
#include <mutex>

#include "wsim_internal.h"

namespace wsim {
namespace {

constexpr int kStaticMaxScenes = 4096;
constexpr int64_t kStaticMaxSegs = int64_t(1) << 18;  // 262,144 packed road-edge segments
constexpr int kMaxDevices = 64;

struct StaticScratch {
    float4 geo[kStaticMaxSegs];
    float inv[kStaticMaxSegs];
    uint8_t flags[kStaticMaxSegs];
    float4 tiles[2 * (kStaticMaxSegs / kTile)];
    float4 sup[kStaticMaxSegs / kTile / kSuper + kStaticMaxScenes];
    uint16_t tperm[kStaticMaxSegs / kTile];
    int32_t seg_off[kStaticMaxScenes + 1];
    int32_t soff[kStaticMaxScenes + 1];
    int32_t seg_cnt[kStaticMaxScenes];
    int32_t order[kStaticMaxScenes];
    int32_t queue;
    int32_t status;
};

// Every GPU that loads the library holds this array (about 6.2 MB) until
// the process exits.  All calls share it.
static __device__ __align__(256) StaticScratch g_scratch;

std::mutex g_mu;
StaticScratch* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device).
int scratch_address(StaticScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return WSIM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return WSIM_ESIZE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return WSIM_ECUDA;
        }
        g_addr[dev] = static_cast<StaticScratch*>(p);
    }
    *out = g_addr[dev];
    return WSIM_OK;
}

// Exclusive prefix sum over one 1024-thread block with a running carry.
__device__ int block_excl_scan(int v, int* wsum, int* carry) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? wsum[warp - 1] : 0) + *carry;
    __syncthreads();
    if (threadIdx.x == 1023) *carry = incl;
    __syncthreads();
    return incl - v;
}

// One CTA, before any kernel reads the roadgraph: checks the CSR offsets
// (agent_off and rg_off start at 0, end at N_tot and R_tot, never decrease)
// and the agents-per-scene limit.  Violations go to the status word, which
// the host reads before the first roadgraph walk.
__global__ void __launch_bounds__(1024) k_static_check(const int32_t* agent_off, const int32_t* rg_off, int S,
                                                       int N_tot, int64_t R_tot, StaticScratch* sc) {
    if (threadIdx.x == 0 &&
        (agent_off[0] != 0 || agent_off[S] != N_tot || rg_off[0] != 0 || rg_off[S] != R_tot))
        atomicCAS(&sc->status, 0, WSIM_EINVAL);
    for (int s = threadIdx.x; s < S; s += 1024) {
        const int n = agent_off[s + 1] - agent_off[s];
        if (n < 0 || rg_off[s + 1] < rg_off[s]) atomicCAS(&sc->status, 0, WSIM_EINVAL);
        if (n > kMaxN) atomicCAS(&sc->status, 0, WSIM_ESIZE);
    }
}

// One CTA: turns the per-scene segment counts into padded segment offsets
// and super-tile offsets and writes the identity work order; packed
// segments beyond the fixed arrays set WSIM_ESIZE.
__global__ void __launch_bounds__(1024) k_static_offsets(int S, StaticScratch* sc) {
    __shared__ int32_t carry[2];
    __shared__ int32_t wsum[32];
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (int base = 0; base < S; base += 1024) {
        const int s = base + threadIdx.x;
        int padded = 0, nsup = 0;
        if (s < S) {
            padded = (sc->seg_cnt[s] + kSegAlign - 1) / kSegAlign * kSegAlign;
            nsup = (padded / kTile + kSuper - 1) / kSuper;
            sc->order[s] = s;
        }
        const int e = block_excl_scan(padded, wsum, &carry[0]);
        const int u = block_excl_scan(nsup, wsum, &carry[1]);
        if (s < S) {
            sc->seg_off[s] = e;
            sc->soff[s] = u;
            if (s == S - 1) {
                sc->seg_off[S] = e + padded;
                sc->soff[S] = u + nsup;
                // packed segments (runs padded to tiles) beyond the fixed arrays
                if (static_cast<int64_t>(e) + padded > kStaticMaxSegs) atomicCAS(&sc->status, 0, WSIM_ESIZE);
            }
        }
    }
}

int read_status(const StaticScratch* sc, cudaStream_t st) {
    int v = 0;
    if (cudaMemcpyAsync(&v, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return WSIM_ECUDA;
    }
    return v;
}

}  // namespace
}  // namespace wsim

using namespace wsim;

extern "C" int wsim_metrics_static(const wsim_config* cfg, const wsim_batch* b, const wsim_state* st,
                                   const wsim_metric_buf* m, int t, void* stream) {
    if (!cfg || !b || !st || !m) return WSIM_EINVAL;
    if (!st->x || !st->y || !st->x_lo || !st->y_lo || !st->th || !st->th_lo || !st->vx || !st->vy)
        return WSIM_EINVAL;
    if (!m->ov || !m->off || !m->logdiv || !m->flags || !m->reward) return WSIM_EINVAL;
    if (!b->agent_off || !b->rg_off || !b->L || !b->W || !b->valid || !b->log_x || !b->log_y) return WSIM_EINVAL;
    if (b->R_tot > 0 && (!b->rg_x || !b->rg_y || !b->rg_poly || !b->rg_type || !b->rg_valid)) return WSIM_EINVAL;
    if (b->S < 1 || b->N_tot < 0 || b->R_tot < 0 || t < 0 || t >= b->T_log) return WSIM_ESIZE;
    // Size limits of the fixed scratch: scenes, and packed segments (a
    // scene of R points has at most R-1 segments, padded to kSegAlign).
    if (b->S > kStaticMaxScenes) return WSIM_ESIZE;
    if (b->R_tot + int64_t(b->S) * (kSegAlign - 1) > kStaticMaxSegs) return WSIM_ESIZE;

    StaticScratch* sc = nullptr;
    int rc = scratch_address(&sc);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: clear the counter and
    // the status word; everything else is rewritten before it is read.
    if (cudaMemsetAsync(&sc->queue, 0, 2 * sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return WSIM_ECUDA;
    }
    // The offsets live in device memory: check them on the device and stop
    // on a violation before any kernel walks a scene's roadgraph range.
    k_static_check<<<1, 1024, 0, s>>>(b->agent_off, b->rg_off, b->S, b->N_tot, b->R_tot, sc);
    if (cudaGetLastError() != cudaSuccess) return WSIM_ECUDA;
    rc = read_status(sc, s);
    if (rc) return rc;
    if (launch_seg_count(b->rg_off, b->rg_x, b->rg_y, b->rg_poly, b->rg_type, b->rg_valid, b->S, sc->seg_cnt, s) !=
        cudaSuccess)
        return WSIM_ECUDA;
    k_static_offsets<<<1, 1024, 0, s>>>(b->S, sc);
    if (cudaGetLastError() != cudaSuccess) return WSIM_ECUDA;
    // The packing kernels rely on the padded total fitting the fixed arrays.
    rc = read_status(sc, s);
    if (rc) return rc;
    if (launch_seg_pack(b->rg_off, b->rg_x, b->rg_y, b->rg_poly, b->rg_type, b->rg_valid, b->S, sc->seg_off,
                        sc->geo, sc->inv, sc->flags, s) != cudaSuccess ||
        launch_tile_build(b->S, sc->seg_off, sc->seg_cnt, sc->geo, sc->flags, sc->tiles, s) != cudaSuccess ||
        launch_tile_order(b->S, sc->seg_off, sc->seg_cnt, sc->tiles, sc->tperm, s) != cudaSuccess ||
        launch_super_build(b->S, sc->seg_off, sc->seg_cnt, sc->soff, sc->tiles, sc->tperm, sc->sup, s) != cudaSuccess)
        return WSIM_ECUDA;

    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.S = b->S;
    a.n_work = b->S;
    a.N_tot = b->N_tot;
    a.T_log = b->T_log;
    a.agent_off = b->agent_off;
    a.L = b->L;
    a.W = b->W;
    a.valid = b->valid;
    a.log_x = b->log_x;
    a.log_y = b->log_y;
    a.segs = Segs{sc->seg_off, sc->seg_cnt, sc->geo, sc->inv, sc->flags, sc->tiles, sc->soff, sc->sup, sc->tperm};
    a.hint = nullptr;  // no nearest-segment cache: bounds come from the tiles
    a.in = CStateP{st->x, st->y, st->x_lo, st->y_lo, st->th, st->th_lo, st->vx, st->vy, st->s, st->s_lo};
    a.m = MetricsP{m->ov, m->off, m->logdiv, m->flags, m->reward};
    a.t_log = t;
    a.do_transition = 0;
    a.do_metrics = 1;
    a.order = sc->order;
    a.queue = &sc->queue;
    a.status = &sc->status;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = b->S < sms * step_blocks_per_sm() ? b->S : sms * step_blocks_per_sm();
    if (launch_step(a, grid, s) != cudaSuccess) return WSIM_ECUDA;
    return read_status(sc, s);
}
