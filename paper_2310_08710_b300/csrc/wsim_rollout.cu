// Scene-resident rollout kernels (sm_103a).
//
// Scenes never exchange data during a rollout, so one CTA can run a scene's
// whole episode (Sec. 5.1, Rollout: T steps of step()) without any global
// synchronisation: the agent state stays in shared memory from step to step
// and only the per-step metrics (and, on request, the per-step states) go to
// global memory.  In the staged shapes one thread copies the scene's packed
// road-edge segments, their flags, culling tiles and super-tiles into shared
// memory with five bulk async copies (TMA) completing on one mbarrier, so
// every off-road query of the episode reads shared memory; scenes too large
// for the stage, and the unstaged shape, read them from global memory (L2).
// CTAs are persistent and take scenes from an atomic counter over a
// cost-ordered work list.  Per step the phases are the same device functions
// as the per-step kernel, so every shape gives bit-identical results.
//
// Launch shapes (threads per CTA x resident CTAs per SM, staged or not) are
// picked per scene-size bucket; wsim_autotune times them on the workload.
// Fewer, larger CTAs keep the same warps per SM with fewer resident scenes,
// whose route and segment data then stay in L2 between steps.
#include "wsim_phases.cuh"

namespace wsim {

// Per-CTA bytes before the stage: the agent block, then the candidate-tile
// caches (list metadata and lists) for cache_n agents, the batch's largest
// scene rounded up to a warp: a batch of small scenes leaves room for more
// resident CTAs.
constexpr size_t kCacheOff = (sizeof(AgentSmem) + 15) / 16 * 16;
__host__ __device__ constexpr size_t agent_bytes(int cache_n) {
    return (kCacheOff + static_cast<size_t>(cache_n) * (kList * sizeof(uint16_t) + sizeof(float4)) + 127) / 128 * 128;
}
constexpr size_t kBytesPerTile = kTile * (16 + 4 + 1) + 32;  // geo + inv + flags + tile records
constexpr size_t kBytesPerSuper = 16;

struct ShapeDesc {
    int threads, min_blocks;
    bool stage;
};
constexpr ShapeDesc kShapes[kRollShapes] = {
    {512, 1, true}, {256, 2, true}, {256, 4, false}, {512, 2, false}, {512, 2, true}};

__device__ __forceinline__ StateP offset_state(const StateP& s, size_t k) {
    return StateP{s.x + k, s.y + k, s.x_lo + k, s.y_lo + k, s.th + k,
                  s.th_lo + k, s.vx + k, s.vy + k, s.s + k, s.s_lo + k};
}

template <int NT, int MINB, bool STAGE, bool DRIVERS>
__global__ void __launch_bounds__(NT, MINB) k_rollout(const StepArgs A) {
    extern __shared__ __align__(128) unsigned char dyn[];
    AgentSmem& sm = *reinterpret_cast<AgentSmem*>(dyn);
    float4* tmeta = reinterpret_cast<float4*>(dyn + kCacheOff);
    uint16_t* tlist = reinterpret_cast<uint16_t*>(tmeta + A.cache_n);
    unsigned char* stage = dyn + agent_bytes(A.cache_n);
    init_cta(sm);
    Counts cnt;
    uint32_t parity = 0;
    const size_t N_tot = static_cast<size_t>(A.N_tot);
    for (;;) {
        if (threadIdx.x == 0) sm.scene = atomicAdd(A.queue, 1);
        __syncthreads();
        const int w = sm.scene;
        if (w >= A.n_work) break;
        const int s = A.order[w];
        const int a0 = A.agent_off[s], N = A.agent_off[s + 1] - a0;
        SegView V = global_view(A.segs, s);
        const bool staged = STAGE && V.nt > 0 && V.nt * kTile <= A.seg_cap;
        if (staged) {
            const int e0 = A.segs.off[s];
            const int ns = V.nt * kTile;
            float4* geo = reinterpret_cast<float4*>(stage);
            float* inv = reinterpret_cast<float*>(geo + ns);
            uint8_t* fl = reinterpret_cast<uint8_t*>(inv + ns);
            float4* tiles = reinterpret_cast<float4*>(fl + ns);
            float4* sup = tiles + 2 * V.nt;
            if (threadIdx.x == 0) {
                const uint32_t bg = ns * 16u, bi = ns * 4u, bf = ns * 1u, bt = V.nt * 32u, bs = V.ns * 16u;
                fence_proxy_async();
                mbar_expect_tx(&sm.bar[0], bg + bi + bf + bt + bs);
                bulk_g2s(geo, A.segs.geo + e0, bg, &sm.bar[0]);
                bulk_g2s(inv, A.segs.inv + e0, bi, &sm.bar[0]);
                bulk_g2s(fl, A.segs.flags + e0, bf, &sm.bar[0]);
                bulk_g2s(tiles, A.segs.tiles + 2 * (e0 / kTile), bt, &sm.bar[0]);
                bulk_g2s(sup, A.segs.sup + A.segs.soff[s], bs, &sm.bar[0]);
            }
            V = SegView{geo, inv, fl, tiles, sup, V.E, V.nt, V.ns, V.perm};  // the order stays in global memory
        }
        load_state<NT>(sm, A, A.in, a0, N);
        for (int j = threadIdx.x; j < 4 * N; j += NT) sm.hint[j] = -1;
        for (int j = threadIdx.x; j < N; j += NT) tmeta[j] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        if (staged) {
            const bool ok = mbar_wait_bounded(&sm.bar[0], parity, kWaitLimitNs);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) set_status(A.status, WSIM_ETIMEOUT);
                mbar_wait_bounded(&sm.bar[0], parity ^ 1u, kWaitLimitNs);
                __syncthreads();
                break;
            }
        }
        if (threadIdx.x == 0) sm.reward = 0;
        __syncthreads();
        // Pipelined steps, two barriers each.  Iteration k: the task phase runs
        // the metrics of state t0+k (k >= 1) together with the transition
        // t0+k -> t0+k+1 (k < T): both read state t0+k and write disjoint
        // arrays.  Warps take the long tasks first (IDM groups, then off-road
        // groups) and the short overlap row pairs last (that order measured
        // fastest); the policy agents follow, one thread each.  The per-agent
        // phase then finishes the metrics of t0+k (row k-1), makes t0+k+1
        // current and prepares its overlap bounds.  The reward of row k-1 is
        // stored at the next task phase.
        for (int k = 0; k <= A.T; ++k) {
            if (k >= 2 && threadIdx.x == 0) {  // reward of row k-2, summed in the last per-agent phase
                A.m.reward[static_cast<size_t>(k - 2) * A.S + s] = sm.reward;
                sm.reward = 0;
            }
            if (k < A.T) {
                transition_idm_tasks(sm, A, a0, N, cnt);
                if (k >= 1) {
                    offroad_tasks(sm, V, sm.hint, tlist, tmeta, N, kListLook * A.p.dt, cnt);
                    row_tasks(sm, N, cnt);
                }
                transition_policy<NT, DRIVERS>(sm, A, A.act ? A.act + static_cast<size_t>(k) * 3 * N_tot : nullptr,
                                      A.t_log + k, a0, N);
            } else {
                offroad_tasks(sm, V, sm.hint, tlist, tmeta, N, kListLook * A.p.dt, cnt);
                row_tasks(sm, N, cnt);
            }
            __syncthreads();
            MetricsP m;
            if (k >= 1) {
                const size_t r = static_cast<size_t>(k - 1) * N_tot;
                m = MetricsP{A.m.ov + r, A.m.off + r, A.m.logdiv + r, A.m.flags + r, nullptr};
            }
            const StateP tr = offset_state(A.traj, static_cast<size_t>(k) * N_tot);
            finish_advance<NT>(sm, A, k >= 1 ? &m : nullptr, A.t_log + k - 1, k < A.T,
                               (k < A.T && A.traj.x) ? &tr : nullptr, a0, N);
            __syncthreads();
        }
        if (threadIdx.x == 0) A.m.reward[static_cast<size_t>(A.T - 1) * A.S + s] = sm.reward;
        store_state<NT>(sm, A.out, a0, N);
        __syncthreads();
    }
    if (DRIVERS) publish_counts(sm, A, cnt);  // the lean kernel's counts are dead code
}

// [0]: the given-action and IDM drivers only (no per-agent driver array),
// without work counting; [1]: every driver, counting on request.
using KernelFn = void (*)(StepArgs);
constexpr KernelFn kKernels[2][kRollShapes] = {
    {k_rollout<512, 1, true, false>, k_rollout<256, 2, true, false>, k_rollout<256, 4, false, false>,
     k_rollout<512, 2, false, false>, k_rollout<512, 2, true, false>},
    {k_rollout<512, 1, true, true>, k_rollout<256, 2, true, true>, k_rollout<256, 4, false, true>,
     k_rollout<512, 2, false, true>, k_rollout<512, 2, true, true>}};

static size_t stage_bytes(int seg_cap) {
    const size_t nt = static_cast<size_t>(seg_cap / kTile);
    return nt * kBytesPerTile + (nt + kSuper - 1) / kSuper * kBytesPerSuper;
}

// Largest stage (in segments, a multiple of kTile) of a shape on this device.
int shape_max_seg_cap(int shape, int cache_n) {
    if (!kShapes[shape].stage) return 0;
    int dev = 0, per_sm = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // per-CTA budget when min_blocks CTAs share the SM (1 KB reserved per CTA)
    size_t budget = static_cast<size_t>(per_sm) / kShapes[shape].min_blocks;
    budget = budget > 1024 ? budget - 1024 : 0;
    if (budget > static_cast<size_t>(optin)) budget = static_cast<size_t>(optin);
    const size_t ab = agent_bytes(cache_n);
    if (budget <= ab + kBytesPerSuper) return 0;
    size_t nt = (budget - ab - kBytesPerSuper) / (kBytesPerTile + kBytesPerSuper / kSuper);
    while (nt > 0 && ab + stage_bytes(static_cast<int>(nt * kTile)) > budget) --nt;
    return static_cast<int>(nt) * kTile;
}

cudaError_t shape_prepare(int shape, int seg_cap, int cache_n, int* blocks_per_sm) {
    const size_t bytes = agent_bytes(cache_n) + stage_bytes(kShapes[shape].stage ? seg_cap : 0);
    int n = 1 << 30;
    for (int d = 0; d < 2; ++d) {
        cudaError_t e = cudaFuncSetAttribute(kKernels[d][shape], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(bytes));
        if (e != cudaSuccess) return e;
        int nd = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nd, kKernels[d][shape], kShapes[shape].threads, bytes);
        if (e != cudaSuccess) return e;
        n = nd < n ? nd : n;
    }
    *blocks_per_sm = n > 0 ? n : 1;
    return cudaSuccess;
}

cudaError_t launch_rollout(int shape, const StepArgs& a, int grid, cudaStream_t st) {
    const size_t bytes = agent_bytes(a.cache_n) + stage_bytes(kShapes[shape].stage ? a.seg_cap : 0);
    kKernels[a.ctrl || a.count ? 1 : 0][shape]<<<grid, kShapes[shape].threads, bytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wsim
