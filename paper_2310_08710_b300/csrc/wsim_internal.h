// Internal types shared by the wsim host API and its kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wsim.h"

namespace wsim {

constexpr int kMaxN = WSIM_MAX_AGENTS;  // agents per scene
constexpr int kThreads = 256;           // threads per step CTA (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 512;             // road-edge segments per staged chunk
constexpr int kSegAlign = 4;            // per-scene segment arrays start on 16 B
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on any mbarrier wait

// Packed road-edge segments of the whole batch (built by wsim_init).
// Scene s owns entries [seg_off[s], seg_off[s] + seg_cnt[s]); seg_off is a
// multiple of kSegAlign and the region is zero-padded up to the next one.
struct Segs {
    const int32_t* off;     // [S+1] padded offsets
    const int32_t* cnt;     // [S]
    const float4* geo;      // (ax, ay, ux, uy): start point and k -> k+1 vector
    const float* inv;       // 1 / |u|^2
    const uint8_t* flags;   // bit0: a segment ends where this one starts; bit1: one starts where it ends
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
};

// Everything one step kernel needs.
struct StepArgs {
    int S, N_tot, T_log;
    const int32_t* agent_off;
    const float *L, *W, *v0;
    const uint8_t *valid, *kind;
    const int32_t* route_off;
    const float *route_x, *route_y;
    const float *log_x, *log_y;
    Segs segs;
    CStateP in;       // state t (transition) or the state measured (metrics only)
    StateP out;       // state t+1 (transition)
    const float* act; // [3][N_tot]
    const uint8_t* ctrl;
    MetricsP m;       // metrics of `out` (or of `in` when do_transition == 0)
    int t_log;        // log row of the metrics
    int do_transition, do_metrics;
    const int32_t* order;  // cost-ordered scene ids
    int32_t* queue;        // scene work counter (zeroed before each launch)
    int32_t* status;       // sticky device status
    unsigned long long* counters;  // [4] work counters (when count != 0)
    int count;
    Params p;
};

// Launchers (kernels.cu).
cudaError_t launch_seg_count(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                             const uint8_t* rg_type, const uint8_t* rg_valid, int S, int32_t* cnt,
                             cudaStream_t st);
cudaError_t launch_seg_pack(const int32_t* rg_off, const float* rg_x, const float* rg_y, const int32_t* rg_poly,
                            const uint8_t* rg_type, const uint8_t* rg_valid, int S, const int32_t* seg_off,
                            float4* geo, float* inv, uint8_t* flags, cudaStream_t st);
cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t st);
cudaError_t launch_plain_scene(const StepArgs& a, int scene, cudaStream_t st);
int step_blocks_per_sm();

}  // namespace wsim
