// Internal types shared by the wsim host API and its kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wsim.h"

namespace wsim {

constexpr int kMaxN = WSIM_MAX_AGENTS;  // agents per scene
constexpr int kStepThreads = 256;       // threads per CTA of the per-step kernels
constexpr int kRollShapes = WSIM_ROLL_SHAPES;  // launch shapes of the scene-resident rollout kernel
constexpr int kBuckets = WSIM_BUCKETS;          // scene-size buckets of the rollout work list
constexpr int kTile = 16;               // road-edge segments per culling tile (half a warp)
constexpr int kSegAlign = kTile;        // per-scene segment arrays start on a tile boundary
constexpr int kMaxSceneSegs = 65536 * kTile;  // packed positions per scene (tile lists hold 16-bit tile indexes)
constexpr int kSuper = 8;               // tiles per super-tile (first culling level)
constexpr int kList = 32;               // tiles in an agent's cached candidate list (one per lane)
constexpr float kSkin = 6.0f;           // extra radius of a candidate list beyond the current need (m)
constexpr float kSkinSmall = 2.0f;      // fallback when the kSkin list would not fit in kList tiles
constexpr float kListLook = 5.0f;       // the wide list is centred this many steps of motion ahead
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on any mbarrier wait
constexpr int kCounters = WSIM_COUNTERS;         // work counters (wsim_counters)

// Packed road-edge segments of the whole batch (built by wsim_init).  Scene s
// owns positions [off[s], off[s] + cnt[s]); off[s] is a multiple of kTile.
// Inside a scene, segments keep roadgraph order and every run of consecutive
// segments (one polyline without a gap) starts on a multiple of kTile; the
// positions between runs and up to the next multiple of kTile hold padding
// (far away, flags 0).  Tile t of the batch covers positions
// [t kTile, (t+1) kTile), i.e. part of one run, and has two float4 records:
// its capsule (chord start, chord) and (radius, 1/|chord|^2, 0, 0).
struct Segs {
    const int32_t* off;    // [S+1]
    const int32_t* cnt;    // [S]
    const float4* geo;     // (ax, ay, ux, uy): start point and k -> k+1 vector
    const float* inv;      // 1 / |u|^2
    const uint8_t* flags;  // bit0: a segment ends where this one starts; bit1: one starts where it ends;
                           // bit2: a segment (0: padding between runs, far away, never nearest)
    const float4* tiles;   // [2 * tiles]
    const int32_t* soff;   // [S+1] first super-tile of each scene
    const float4* sup;     // super-tile bounding boxes: super-tile j of scene s covers its tiles
                           // tperm[8j .. 8j+7]
    const uint16_t* tperm; // [tiles] per scene: its tiles in super-tile order (scene-relative indexes,
                           // sorted along a Morton curve of the tile centres so that a super-tile is
                           // compact); null: identity
};

struct StateP {
    float *x, *y, *x_lo, *y_lo, *th, *th_lo, *vx, *vy, *s, *s_lo;
};
struct CStateP {
    const float *x, *y, *x_lo, *y_lo, *th, *th_lo, *vx, *vy, *s, *s_lo;
};

struct MetricsP {
    float *ov, *off, *logdiv;
    uint8_t* flags;
    int32_t* reward;
};

struct Params {
    float dt, amax, b, T, s0, dq, h, inv_h, gap_min, idm_sqrt_ab2;  // 2 sqrt(a b)
    float inv_dt;                      // 1 / dt, rounded once
    float kin_amax, kin_kmax;  // kinematic infeasibility limits
    float da_max, dk_max, dd_max, dt_max;  // discrete action grids (ranges)
    int na, nk, nd, nt;                    // ... and values per component
};

// Everything a step or rollout kernel needs.
struct StepArgs {
    int S, N_tot, T_log;
    int n_work;       // scenes in the work list `order`
    const int32_t* agent_off;
    const float *L, *W, *v0;
    const uint8_t *valid, *kind;
    const int32_t* route_off;
    const float *route_x, *route_y;
    const float* route_rf;  // per agent: its route's largest segment length over route_h (+inf if not finite)
    const float *log_x, *log_y;
    const float *log_th, *log_vx, *log_vy;  // may be null (no expert, no log playback)
    Segs segs;
    int32_t* hint;    // [N_tot][4] nearest-segment cache of the per-step kernels (may be null)
    uint16_t* tlist;  // [N_tot][kList] candidate-tile cache of the per-step kernels (may be null)
    float4* tmeta;    // [N_tot] (centre x, centre y, radius, count) of each candidate list
    CStateP in;       // state t (transition) or the state measured (metrics only)
    StateP out;       // state t+1 (per-step) / final state (rollout)
    const float* act; // [3][N_tot] (per step) or [T][3][N_tot] (rollout)
    const uint8_t* ctrl;
    MetricsP m;       // metrics of `out` (or of `in` when do_transition == 0); rollout: [T][...]
    int t_log;        // log row of the metrics (rollout: of the first step)
    int T;            // rollout steps (scene-resident kernel)
    StateP traj;      // rollout: states of every step, [T][N_tot] blocks (x == nullptr: none)
    int do_transition, do_metrics;
    const int32_t* order;  // cost-ordered scene ids
    int32_t* queue;        // scene work counter (zeroed before each launch)
    int32_t* status;       // sticky device status
    unsigned long long* counters;  // [kCounters] work counters (when count != 0)
    int count;
    int seg_cap;           // rollout: segments that fit in the shared-memory stage
    int cache_n;           // rollout: agents of the per-CTA candidate-tile caches (>= every scene's N)
    Params p;
};

// Launchers (wsim_kernels.cu, wsim_rollout.cu).
cudaError_t launch_seg_count(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                             const uint8_t* rg_type, const uint8_t* rg_valid, int S, int32_t* cnt,
                             cudaStream_t st);
cudaError_t launch_seg_pack(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                            const uint8_t* rg_type, const uint8_t* rg_valid, int S, const int32_t* seg_off,
                            float4* geo, float* inv, uint8_t* flags, cudaStream_t st);
cudaError_t launch_tile_build(int S, const int32_t* seg_off, const int32_t* seg_cnt, const float4* geo,
                              const uint8_t* flags, float4* tiles, cudaStream_t st);
// Super-tile order of each scene's tiles (Morton order of the tile centres;
// the identity for scenes of more than kOrderMaxTiles tiles).
constexpr int kOrderMaxTiles = 4096;
cudaError_t launch_tile_order(int S, const int32_t* seg_off, const int32_t* seg_cnt, const float4* tiles,
                              uint16_t* tperm, cudaStream_t st);
cudaError_t launch_super_build(int S, const int32_t* seg_off, const int32_t* seg_cnt, const int32_t* soff,
                               const float4* tiles, const uint16_t* tperm, float4* sup, cudaStream_t st);
cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t st);
// route_rf[g] = (largest segment length of agent g's route) / route_h,
// rounded up; +inf when a segment length is not finite; 0 without segments.
cudaError_t launch_route_speed(const int32_t* route_off, const float* rx, const float* ry, int N, float inv_h,
                               float* rf, cudaStream_t st);
// Discrete actions: continuous [T][3][N_tot] <-> flat grid indices [T][N_tot].
cudaError_t launch_discretize(const StepArgs& a, const float* act, int T, int32_t* idx, cudaStream_t st);
cudaError_t launch_decode_actions(const StepArgs& a, const int32_t* idx, int T, float* act, cudaStream_t st);
// Open-loop expert actions over log rows [t0, t0+T] into act [T][3][N_tot].
cudaError_t launch_expert_actions(const StepArgs& a, int t0, int T, float* act, cudaStream_t st);
cudaError_t launch_plain_scene(const StepArgs& a, int scene, cudaStream_t st);
int step_blocks_per_sm();
// Scene-resident rollout, launch shapes (threads x CTAs per SM, stage): 0
// 512 x 1 large stage, 1 256 x 2 small stage, 2 256 x 4 no stage, 3 512 x 2
// no stage, 4 512 x 2 small stage.  seg_cap: staged segments (a.seg_cap at
// launch).
// cache_n: agents of the per-CTA candidate-tile caches (a.cache_n at launch).
int shape_max_seg_cap(int shape, int cache_n);
cudaError_t shape_prepare(int shape, int seg_cap, int cache_n, int* blocks_per_sm);
cudaError_t launch_rollout(int shape, const StepArgs& a, int grid, cudaStream_t st);
// Observation (wsim_observe.cu): roadgraph point tiles of at most kPtTile
// consecutive points of one polyline run per scene (counted per scene, then
// their starts written; tile t holds points pt_start[t] .. pt_start[t+1]-1),
// their boxes, and the per-observer kernels.
constexpr int kPtTile = 32;
cudaError_t launch_pt_count(const int32_t* rg_off, const int32_t* rg_poly, int S, int32_t* tiles_per_scene,
                            cudaStream_t st);
cudaError_t launch_pt_tiles(const int32_t* rg_off, const int32_t* rg_poly, const int32_t* tile_off, const float* rg_x,
                            const float* rg_y, const uint8_t* rg_valid, int S, int32_t* pt_start, float4* box,
                            int32_t* cnt, cudaStream_t st);
cudaError_t launch_observe(const StepArgs& a, const uint8_t* observers, int32_t* list, int32_t* count,
                           const float* rg_x, const float* rg_y, const uint8_t* rg_valid, const int32_t* tile_off,
                           const int32_t* pt_start, const float4* box, const int32_t* cnt, const int32_t* scene_of,
                           int M, int K, float* agents, uint8_t* agents_valid, float* rg, int32_t* rg_idx,
                           cudaStream_t st);
// Route metrics (wsim_route.cu).
cudaError_t launch_route(const StepArgs& a, const int32_t* path_off, const int32_t* path_pt_off, const float* path_x,
                         const float* path_y, const uint8_t* path_on, float max_dist, float max_rel, float* progress,
                         uint8_t* off_route, cudaStream_t st);
// Backpropagation through the rollout (wsim_bptt.cu).
cudaError_t launch_bptt(const StepArgs& a, float* ckpt, float* segbuf, int ck, double* loss, float* dact,
                        float lambda, float tau, int grid, bool plain, cudaStream_t st);
// Recording forward (checkpoints, loss, metric rows and their deciding
// indices) and the backward of a weighted objective of its metrics and loss.
cudaError_t launch_record(const StepArgs& a, float* ckpt, int ck, double* loss, int metrics, int16_t* rec_ov,
                          int32_t* rec_off, float lambda, float tau, int grid, cudaStream_t st);
cudaError_t launch_backward(const StepArgs& a, float* ckpt, float* segbuf, int ck, const int16_t* rec_ov,
                            const int32_t* rec_off, const float* g_logdiv, const float* g_ov, const float* g_off,
                            const double* loss_w, float* dact, const StateP& dst0, float lambda, float tau, int grid,
                            cudaStream_t st);
int bptt_blocks_per_sm(int which = 0);

}  // namespace wsim
