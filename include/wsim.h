/*
 * wsim: batched closed-loop driving-simulator step on one B300 (sm_103a).
 *
 * C ABI of libwsim.so.  It implements the data-parallel hot path of the
 * Waymax simulator (arXiv 2310.08710): per agent, bicycle and delta dynamics
 * (App. A.1) and IDM route-following sim agents (Sec. 3.5); per scene, the
 * pairwise rotated-box overlap (Sec. 3.4, collision), the signed distance of
 * each box corner to the oriented road edges (Sec. 3.4, off-road), the log
 * divergence (Sec. 3.4, displacement error) and the sparse reward (Sec. 5.2);
 * an 80-step rollout (Sec. 5.1, Rollout) and its adjoint for BPTT (the
 * differentiable simulation of Sec. 6).
 *
 * Calling conventions shared by every entry point
 * -----------------------------------------------
 *  - Pointers named in the structs below are DEVICE pointers into memory the
 *    caller owns (e.g. torch tensors).  The library never frees them and keeps
 *    no reference to them after a call returns, except the scene batch given
 *    to wsim_init, which must stay alive and unchanged until wsim_destroy.
 *  - Layouts are structure-of-arrays of float32 / int32 / uint8.  Agents and
 *    roadgraph points are in CSR form over scenes (agent_off, rg_off).
 *    Per-step arrays are indexed by the global agent index g in [0, N_tot).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls enqueue work and return without synchronising, except
 *    wsim_init, wsim_status and wsim_destroy, which synchronise the stream.
 *  - Every call returns WSIM_OK (0) or a negative WSIM_E* code.  Errors found
 *    on the host (bad sizes, null pointers) are returned before any work is
 *    enqueued.  Errors found on the device (non-finite input, a bounded wait
 *    that expired) are recorded in a sticky status word that wsim_status
 *    reads; no kernel traps.
 *  - A context may be used from one host thread at a time.
 */
#ifndef WSIM_H
#define WSIM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WSIM_OK 0
#define WSIM_EINVAL (-1)      /* null pointer, bad enum, inconsistent CSR       */
#define WSIM_ESIZE (-2)       /* a size beyond the documented limits            */
#define WSIM_ECUDA (-3)       /* a CUDA runtime call failed                      */
#define WSIM_ENONFINITE (-4)  /* a non-finite action or state reached a kernel   */
#define WSIM_ETIMEOUT (-5)    /* a bounded device-side wait gave up              */
#define WSIM_ENOMEM (-6)      /* device allocation failed                        */
#define WSIM_ESTATE (-7)      /* call out of order (e.g. backward before rollout)*/

#define WSIM_MAX_AGENTS 256   /* agents per scene                                */
#define WSIM_LOOKAHEAD 32     /* IDM look-ahead samples (one per warp lane)      */

/* Agent kinds. */
#define WSIM_KIND_BICYCLE 0   /* policy agent, action (a [m/s^2], kappa [1/m])    */
#define WSIM_KIND_DELTA 1     /* policy agent, action (dx [m], dy [m], dtheta)    */
#define WSIM_KIND_IDM 2       /* IDM sim agent following its route               */

/* Roadgraph point types: only RG_EDGE points form road-edge segments. */
#define WSIM_RG_EDGE 1

/* Metric flag bits (wsim_metric_buf.flags). */
#define WSIM_FLAG_COLLISION 1
#define WSIM_FLAG_OFFROAD 2
#define WSIM_FLAG_KININF 4    /* kinematically infeasible transition (Sec. 3.4)  */

/* Who drives an agent in a step (the per-agent ctrl array; NULL ctrl means
 * WSIM_CTRL_ACTION for every agent). */
#define WSIM_CTRL_HOLD 0      /* policy agent keeps its state                    */
#define WSIM_CTRL_ACTION 1    /* policy agent takes the given action             */
#define WSIM_CTRL_EXPERT 2    /* policy agent takes the expert action (Sec. 5.2) */
#define WSIM_CTRL_LOG 3       /* any agent replays the log (Sec. 3.5)            */
#define WSIM_CTRL_EXPERT_DISCRETE 4 /* policy agent: the expert action snapped to
                                       the discrete grid (Sec. 5.2)              */

/* Rollout modes. */
#define WSIM_MODE_GRAPH 0      /* persistent step kernel per step, CUDA graph   */
#define WSIM_MODE_STREAM 1     /* persistent step kernel per step, no graph     */
#define WSIM_MODE_PLAIN 2      /* one launch per scene per phase (baseline)     */
#define WSIM_MODE_FUSED 3      /* one scene-resident launch for all T steps     */

/* Method constants.  wsim_default_config fills the values used throughout. */
typedef struct {
    float dt;          /* step length [s]: 0.1 (Sec. 3.1, 10 Hz)                 */
    float idm_amax;    /* IDM maximum acceleration a [m/s^2]: 2.0                */
    float idm_b;       /* IDM comfortable deceleration b [m/s^2]: 3.0            */
    float idm_T;       /* IDM time headway T [s]: 1.5                            */
    float idm_s0;      /* IDM minimum gap s0 [m]: 2.0                            */
    float idm_dq;      /* spacing of the look-ahead samples along the route [m]: 2 */
    float route_h;     /* parameter length of one route segment [m]: 0.5         */
    float gap_min;     /* lower clamp of the bumper gap [m]: 0.1                 */
    float loss_lambda; /* weight of the overlap penalty in the BPTT loss: 1.0    */
    float loss_tau;    /* softplus temperature of the overlap penalty [m]: 0.25  */
    int32_t ckpt_every;/* BPTT checkpoint interval in steps (1 = store all): 10  */
    int32_t tile_segs; /* road-edge segments per culling tile (0 = default)      */
    float kin_amax;    /* kinematic infeasibility: |a| limit [m/s^2]: 6 (Sec. 3.4) */
    float kin_kmax;    /* ... |kappa| limit [1/m]: 0.3 (Sec. 3.4)                 */
    float route_max_dist; /* off-route: farther than this from every on-route path [m]: 5 */
    float route_max_rel;  /* off-route: an off-route path nearer by more than this [m]: 2 */
    /* Discrete action spaces (Sec. 5.2): n uniform values over [-max, max]
     * per component.  Bicycle: a 13 over 6 m/s^2, kappa 31 over 0.3 1/m;
     * delta: dx and dy 25 over 6 m, dtheta 13 over 0.3 rad. */
    float disc_a_max, disc_k_max, disc_d_max, disc_t_max;
    int32_t disc_na, disc_nk, disc_nd, disc_nt;
} wsim_config;

/* A batch of S scenes (all device pointers; sizes on the host).
 * Scene s owns agents [agent_off[s], agent_off[s+1]) and roadgraph points
 * [rg_off[s], rg_off[s+1]).  Agent g owns route points [route_off[g],
 * route_off[g+1]) (>= 2 for IDM agents, may be empty otherwise).  Logs are
 * time-major [T_log][N_tot].  Points k and k+1 of a scene form a road-edge
 * segment, oriented k -> k+1, iff both are valid, both have type
 * WSIM_RG_EDGE and both carry the same polyline id (Sec. 3.4, off-road: the
 * road lies on the left of an oriented edge). */
typedef struct {
    int32_t S, N_tot, T_log, pad_;
    int64_t R_tot;                     /* roadgraph points in the batch       */
    int64_t route_tot;                 /* route points in the batch           */
    const int32_t *agent_off, *rg_off; /* [S+1]                               */
    const float *L, *W, *idm_v0;       /* [N_tot] box length, width; IDM v0   */
    const uint8_t *valid, *kind;       /* [N_tot]                             */
    const int32_t *route_off;          /* [N_tot+1]                           */
    const float *route_x, *route_y;    /* [route_tot]                         */
    const float *rg_x, *rg_y;          /* [R_tot]                             */
    const int32_t *rg_poly;            /* [R_tot] polyline id                 */
    const uint8_t *rg_type, *rg_valid; /* [R_tot]                             */
    const float *log_x, *log_y;        /* [T_log][N_tot] logged positions     */
    const float *log_th;               /* [T_log][N_tot] logged heading; with */
    const float *log_vx, *log_vy;      /* the logged velocity it may be NULL, */
                                       /* which disables the expert and log   */
                                       /* playback (WSIM_EINVAL if asked for) */
    /* Route paths of each scene's first agent (Sec. 3.2 on-/off-route paths;
     * may be NULL: no route metrics): scene s owns paths [path_off[s],
     * path_off[s+1]), path p owns points [path_pt_off[p], path_pt_off[p+1]),
     * path_on[p] = 1 marks an on-route path. */
    const int32_t *path_off;           /* [S+1]                               */
    const int32_t *path_pt_off;        /* [paths+1]                           */
    const float *path_x, *path_y;      /* [path points]                       */
    const uint8_t *path_on;            /* [paths]                             */
} wsim_batch;

/* Agent state, [N_tot] each.  Positions, heading and route cursor are
 * float32 pairs (hi, lo) whose exact sum is the value (compensated
 * summation keeps positions near 400 m inside 1e-5 m).  s is the arc-length
 * parameter of an IDM agent on its route (unused by policy agents). */
typedef struct {
    float *x, *y, *x_lo, *y_lo, *th, *th_lo, *vx, *vy, *s, *s_lo;
} wsim_state;

/* Per-step metrics.  ov: largest SAT overlap depth against another valid
 * agent (> 0 = collision; -inf if none).  off: largest signed distance of a
 * box corner to the nearest road edge (> 0 = off road; -inf if the scene has
 * no edge).  logdiv: distance to the logged position.  flags: bit0 collision,
 * bit1 off road, bit2 kinematically infeasible transition into this state
 * (Sec. 3.4: the App. A.1 bicycle inverse kinematics of the two consecutive
 * states, direction atan2(vy', vx') against the old heading, breaks |a| <=
 * kin_amax or |kappa| <= kin_kmax; set by wsim_step and wsim_rollout, 0 from
 * wsim_metrics, which sees one state).  reward[s] = -(collisions + off-road
 * agents) of scene s.
 * Invalid agents report 0 everywhere.  In wsim_rollout each pointer is the
 * base of a [T][N_tot] (reward [T][S]) array. */
typedef struct {
    float *ov, *off, *logdiv;
    uint8_t *flags;
    int32_t *reward;
} wsim_metric_buf;

typedef struct wsim_ctx wsim_ctx;

/* Fills *cfg with the default constants listed in wsim_config. */
void wsim_default_config(wsim_config *cfg);

/* reset() of Sec. 4 (the initialisation half): validates the batch, builds
 * the packed road-edge segments and their culling tiles on the device and
 * the cost-ordered scene work list.  Allocates device scratch owned by the
 * context.  Synchronises `stream`.  Limits: agents per scene <=
 * WSIM_MAX_AGENTS, S >= 1, T_log >= 2; a scene's road-edge segments, each
 * polyline run padded to a multiple of 16, at most 2^20 positions, and the
 * batch's at most INT32_MAX once every scene is padded to a multiple of 16
 * (else WSIM_ESIZE). */
int wsim_init(wsim_ctx **out, const wsim_config *cfg, const wsim_batch *b, void *stream);

/* step() of Sec. 4: state t -> t+1 for every scene, then the metrics of t+1
 * against log row t+1.  act is [3][N_tot]: (a, kappa, unused) for bicycle
 * agents, (dx, dy, dtheta) for delta agents; IDM agents ignore it.
 * ctrl [N_tot] (device, may be NULL = all WSIM_CTRL_ACTION) picks the driver
 * of each agent: a policy agent holds its state (WSIM_CTRL_HOLD), takes its
 * action (WSIM_CTRL_ACTION), or takes the expert action (WSIM_CTRL_EXPERT:
 * the App. A.1 inverse of its action space from its state t to log row t+1,
 * then its forward dynamics); any agent with WSIM_CTRL_LOG takes log row t+1
 * as its state; WSIM_CTRL_EXPERT_DISCRETE snaps the expert action to the
 * discrete grid (see wsim_discretize) before applying it; IDM agents follow
 * their route for every value but WSIM_CTRL_LOG.
 * Invalid agents keep their state.  A value above WSIM_CTRL_EXPERT_DISCRETE, or the
 * expert or log playback without log_th/log_vx/log_vy, holds the agent and
 * sets the device status to WSIM_EINVAL.  `in` and `out` must not alias.
 * m may be NULL (transition only).  Requires 0 <= t and t+1 < T_log. */
int wsim_step(wsim_ctx *ctx, const wsim_state *in, const float *act, const uint8_t *ctrl,
              wsim_state *out, const wsim_metric_buf *m, int t, void *stream);

/* The metrics of state st against log row t (Sec. 3.4). */
int wsim_metrics(wsim_ctx *ctx, const wsim_state *st, const wsim_metric_buf *m, int t, void *stream);

/* Rollout (Sec. 5.1): T steps from time index t0.  st holds state t0 on
 * entry and state t0+T on return (device order); act_seq is [T][3][N_tot]
 * (may be NULL only with a ctrl array in which no agent takes
 * WSIM_CTRL_ACTION); ctrl as in wsim_step, for every step;
 * mseq arrays are [T][N_tot] ([T][S] for reward), row k holding the metrics
 * of time t0+k+1.  mode: WSIM_MODE_FUSED (fastest) runs one persistent
 * launch in which each CTA carries whole scenes through all T steps with
 * the state and the scene's road-edge segments resident in shared memory;
 * WSIM_MODE_GRAPH replays a CUDA graph of T per-step launches (captured on
 * the first call and re-captured when pointers or T change);
 * WSIM_MODE_STREAM launches the same per-step kernels directly;
 * WSIM_MODE_PLAIN launches one kernel per scene and phase.  All four give
 * bit-identical results.  traj (may be NULL) receives the states of times
 * t0+1..t0+T as [T] consecutive wsim_state-shaped blocks: traj[k] pointers
 * are the base pointers advanced by k*N_tot. */
int wsim_rollout(wsim_ctx *ctx, wsim_state *st, const float *act_seq, const uint8_t *ctrl, int t0,
                 int T, int mode, const wsim_metric_buf *mseq, const wsim_state *traj, void *stream);

/* Route metrics (Sec. 3.4) of each scene's first agent at state st:
 * progress[s] (device, [S]) = (d_x - d_p) / (d_q - d_p), where d_x is the
 * arc length along the on-route path nearest to the agent (ties: the lower
 * path) of the agent's nearest point on it (ties: the lower segment), and
 * d_p, d_q those of the first and last logged positions (log rows 0 and
 * T_log-1) on the same path; NaN when d_q - d_p <= 1 mm or the scene has no
 * on-route path.  off_route[s] (device, [S]) = 1 when the agent is farther
 * than route_max_dist from every on-route path or nearer to an off-route
 * path by more than route_max_rel.  Requires the batch's route paths
 * (WSIM_EINVAL without).  Asynchronous on `stream`. */
int wsim_route_metrics(wsim_ctx *ctx, const wsim_state *st, float *progress, uint8_t *off_route, void *stream);

/* Discrete action spaces (Sec. 5.2: the expert of a discrete action space
 * discretises the continuous inverse).  A component value v on a grid of n
 * values over [-max, max] has index rint(fl(v / step) + c) clamped to
 * [0, n-1], step = fl(2 max / (n-1)), c = (n-1)/2 (float32), and the grid
 * value of index i is fl((i - c) * step).  Flat indices: bicycle
 * i_a * disc_nk + i_k; delta (i_x * disc_nd + i_y) * disc_nt + i_t.
 * wsim_discretize: act [T][3][N_tot] -> idx [T][N_tot] (-1 for IDM and
 * invalid agents).  wsim_decode_actions: idx -> act [T][3][N_tot] (grid
 * values; zeros for idx < 0; an index past the grid also gives zeros and
 * sets WSIM_EINVAL in the device status).  Device arrays, caller-owned;
 * asynchronous on `stream`. */
int wsim_discretize(wsim_ctx *ctx, const float *act, int T, int32_t *idx, void *stream);
int wsim_decode_actions(wsim_ctx *ctx, const int32_t *idx, int T, float *act, void *stream);

/* Expert actions, open loop (Sec. 5.2: the inverse of each agent's action
 * space fitted to the logged trajectory, App. A.1): act_out [T][3][N_tot]
 * (device, caller-owned) row k receives the action that takes log row
 * t0+k to log row t0+k+1: (a, kappa, 0) for bicycle agents by the inverse
 * kinematics, (dx, dy, dtheta) for delta agents, 0 for IDM and invalid
 * agents.  Float32: the direction within 4e-7 rad (the library's own
 * atan2), a within an ulp of (|v'| - |v|) / dt, kappa = turn / distance
 * within 2 ulps.  Requires log_th/log_vx/log_vy (else WSIM_EINVAL), 0 <= t0,
 * T >= 0 and t0+T < T_log (else WSIM_ESIZE).  Asynchronous on `stream`. */
int wsim_expert_actions(wsim_ctx *ctx, int t0, int T, float *act_out, void *stream);

/* Observation (Sec. 3.2: each agent sees the other agents in its own frame
 * and the roadgraph subsampled by distance) of state st, for every agent g
 * with observers[g] != 0 (device [N_tot]; NULL: every valid agent).  The
 * frame of g has its origin at g's centre and its x axis along g's heading.
 * agents [N_tot][M][5] (device, caller-owned): agent j of g's scene (index
 * within the scene) as (x, y, yaw, vx, vy) in g's frame, yaw reduced to
 * [-pi, pi]; agents_valid [N_tot][M]: 1 iff agent j is valid and not g.
 * rg [N_tot][K][2] and rg_idx [N_tot][K]: the K valid roadgraph points
 * (any type) of g's scene nearest to g's centre, ascending, ties to the
 * lower global point index, as (x, y) in g's frame and their global index;
 * -1 and 0 past the scene's valid points.  Ranking key (float32, exact
 * integer decisions): c = fl(x + x_lo), d = fl(p - c), key =
 * fmaf(dx, dx, dy*dy).  Rows of other agents are not written.  Requires
 * M >= the largest scene's agent count and 1 <= K <= WSIM_OBS_MAX_K (else
 * WSIM_ESIZE); more than WSIM_OBS_MAX_K points at the K-th key set
 * WSIM_ESIZE in the device status and leave that observer's points at -1.
 * The first call builds the context's roadgraph point tiles (allocation,
 * synchronises `stream`); later calls are asynchronous. */
#define WSIM_OBS_MAX_K 4096
int wsim_observe(wsim_ctx *ctx, const wsim_state *st, const uint8_t *observers, int M, int K, float *agents,
                 uint8_t *agents_valid, float *rg, int32_t *rg_idx, void *stream);

/* Launch configuration of the scene-resident rollout (WSIM_MODE_FUSED).
 * Five launch shapes exist (threads per CTA x CTAs per SM, where the
 * scene's road-edge segments are read from): 0 = 512 x 1, large
 * shared-memory stage; 1 = 256 x 2, small stage; 2 = 256 x 4, global memory
 * (L2); 3 = 512 x 2, global memory; 4 = 512 x 2, small stage.  Scenes are
 * grouped at wsim_init into size buckets by road-edge segment count: bucket
 * 0 fits the small stage, bucket 1 the large one, bucket 2 neither.  Either
 * one shape runs the whole cost-ordered batch (split = 0, single_shape) or
 * each bucket runs its own shape on its own stream, concurrently (split = 1,
 * bucket_shape).  A staged shape reads a scene that does not fit its stage
 * from global memory.  Every configuration gives bit-identical results. */
#define WSIM_ROLL_SHAPES 5
#define WSIM_BUCKETS 3
typedef struct {
    int32_t split;            /* 0: one launch of single_shape; 1: per bucket   */
    int32_t single_shape;
    int32_t bucket_shape[WSIM_BUCKETS];
    int32_t bucket_scenes[WSIM_BUCKETS]; /* filled by wsim_get_tuning / wsim_autotune */
    float ms_single[WSIM_ROLL_SHAPES];   /* wsim_autotune: T-step time of each shape */
    float ms_bucket[WSIM_BUCKETS][WSIM_ROLL_SHAPES]; /* ... of each shape on each bucket alone (-1: n/a) */
    float ms_split;           /* ... of the split configuration (-1: n/a)       */
} wsim_tuning;

/* Autotuner: times a T-step rollout from state st (copied; st is not
 * modified) for each single shape, for each shape on each non-empty bucket,
 * and for the split configuration built from the best shape of each bucket,
 * after one warm-up run each; keeps the fastest configuration for later
 * WSIM_MODE_FUSED rollouts and reports all times in *out.  Allocates and
 * frees scratch for the metric rows; synchronises `stream`. */
int wsim_autotune(wsim_ctx *ctx, const wsim_state *st, const float *act_seq, int t0, int T, wsim_tuning *out,
                  void *stream);

/* Set a configuration (e.g. one saved from an earlier wsim_autotune; only
 * split, single_shape and bucket_shape are read) / read the current one. */
int wsim_set_tuning(wsim_ctx *ctx, const wsim_tuning *t);
int wsim_get_tuning(wsim_ctx *ctx, wsim_tuning *out);

/* Backpropagation through a whole rollout (the differentiable simulation of
 * Sec. 6).  Loss of scene s:
 *   L_s = sum_{t=t0+1}^{t0+T} sum_i d_i(t)^2
 *         + loss_lambda * sum_t sum_{i<j} loss_tau * softplus(d_ij(t) / loss_tau)
 * over valid agents, d_i = distance to the logged position, d_ij = SAT
 * overlap depth (> 0 when overlapping).  Runs the T-step rollout from st0
 * (not modified; all policy agents controlled) with the loss, storing the
 * state every ckpt_every steps, then the reverse sweep, recomputing each
 * segment from its checkpoint.  loss[S] (device, float64) receives L_s; dact
 * (device, [T][3][N_tot], may be NULL for the loss only) receives dL/dact
 * for bicycle (a, kappa, 0) and delta (dx, dy, dtheta) agents and 0 for the
 * others.  IDM agents move as in wsim_rollout but are constants for the
 * derivative.  Results do not depend on ckpt_every (bit-identical) and use
 * no float atomics.  flags: WSIM_GRAD_PLAIN launches one kernel per scene
 * (baseline) instead of the persistent kernel.  Grows the context's
 * checkpoint scratch on first use (synchronising `stream` then). */
#define WSIM_GRAD_PLAIN 1
int wsim_loss_grad(wsim_ctx *ctx, const wsim_state *st0, const float *act_seq, int t0, int T, int ckpt_every,
                   int flags, double *loss, float *dact, void *stream);

/* Differentiable rollout (the differentiable simulation of Sec. 6), forward
 * half.  Runs the T-step rollout from st0 (not modified) with every policy
 * agent taking act_seq ([T][3][N_tot], as wsim_rollout with ctrl NULL; IDM
 * agents follow their routes) and keeps a record of it in the context: the
 * state every ckpt_every steps and, when mseq is given, the indices that
 * decided each step's metrics: per valid agent the partner of its deepest
 * overlap (exact maximum, ties to the lower index) and the corner, road-edge
 * segment and side of its largest off-road distance (ties to the lower
 * corner).  mseq (may be NULL: no metrics) receives the metric rows exactly
 * as wsim_rollout writes them (bit for bit); loss (device float64 [S], may be
 * NULL) the scene losses of wsim_loss_grad; st_T (may be NULL, must not alias
 * st0) the state at t0+T.  A context holds one record: a new call replaces
 * it.  The record's scratch grows on first use and when T grows (the call
 * then synchronises `stream`); otherwise asynchronous. */
int wsim_rollout_record(wsim_ctx *ctx, const wsim_state *st0, const float *act_seq, int t0, int T, int ckpt_every,
                        const wsim_metric_buf *mseq, double *loss, wsim_state *st_T, void *stream);

/* Weights of the per-step metrics in the objective of wsim_rollout_backward:
 * device float32 [T][N_tot] arrays, row k for time t0+k+1 (the rows of the
 * recorded rollout's mseq); NULL = all 0. */
typedef struct {
    const float *logdiv, *ov, *off;
} wsim_metric_grad;

/* Differentiable rollout, reverse half: the gradient of
 *   J = sum_s loss_w[s] L_s
 *     + sum_k sum_g ( gm.logdiv[k][g] logdiv_g + gm.ov[k][g] ov_g + gm.off[k][g] off_g )
 * over the recorded rollout, with respect to its actions and its initial
 * state.  L_s is the loss of wsim_loss_grad; logdiv, ov and off are the
 * metric rows of the recorded rollout (App. A.1 dynamics, Sec. 3.4 metrics).
 * ov and off are maxima: their derivative is that of the recorded deciding
 * pair or corner (the nearest point on the recorded segment, the side fixed);
 * a metric of -inf (no other valid agent, no road edge) and every metric of
 * an invalid agent add nothing.  IDM agents move but are constants for the
 * derivative.  act_seq: the recorded rollout's actions, unchanged.  loss_w
 * (device float64 [S], may be NULL = no loss term); gm may be NULL (no metric
 * term).  dact ([T][3][N_tot], may be NULL) receives dJ/dact as
 * wsim_loss_grad writes it; dst0 (may be NULL, not both) receives dJ/d(state
 * t0): x and x_lo both hold dJ/dx of x = x + x_lo (likewise y, th), vx and vy
 * their derivatives, s and s_lo 0.  The segments between checkpoints are
 * recomputed with the forward's code, so results do not depend on
 * ckpt_every; no float atomics (deterministic).  WSIM_ESTATE without a
 * record, or with metric weights for a record made without mseq.
 * Asynchronous on `stream`. */
int wsim_rollout_backward(wsim_ctx *ctx, const float *act_seq, const wsim_metric_grad *gm, const double *loss_w,
                          float *dact, wsim_state *dst0, void *stream);

/* Sticky device status: synchronises `stream`, writes the first device error
 * code recorded since the last call (WSIM_OK if none) to *device_status and
 * clears it. */
int wsim_status(wsim_ctx *ctx, int *device_status, void *stream);

/* Work counters summed over the launches since wsim_set_counting(ctx, 1)
 * (for roofline accounting; 0 when counting is off): [0] corner-segment
 * distance evaluations, [1] culling-tile bound tests, [2] SAT pair
 * evaluations (each unordered pair counts 2; in wsim_loss_grad and
 * wsim_rollout_backward those of the loss and its adjoint), [3] IDM
 * look-ahead sample-box tests, [4] overlap pair bound tests, [5] IDM
 * lead-candidate circle tests.  Synchronises. */
#define WSIM_COUNTERS 6
int wsim_set_counting(wsim_ctx *ctx, int on);
int wsim_counters(wsim_ctx *ctx, int64_t out[WSIM_COUNTERS], void *stream);

/* Message for a WSIM_E* code. */
const char *wsim_strerror(int code);

/* Frees the context's device scratch; synchronises its last stream. */
void wsim_destroy(wsim_ctx *ctx);

/* Metrics of state st against log row t, like wsim_metrics, but with no
 * context and no device allocation at all.  The paper has no counterpart;
 * this is for callers that cannot call cudaMalloc when they need the metrics
 * (a caching allocator or fixed arena that owns all device memory, code that
 * must not allocate).  The scratch wsim_init would allocate lives instead in
 * one file-scope device array of about 6.2 MB that every GPU loading the
 * library holds until the process exits.  Limits: at most 4096 scenes, and
 * at most 262144 packed road-edge positions (segments, with each run of
 * consecutive segments padded to a multiple of 16 and each scene to a
 * multiple of 16; R_tot + 15 * S > 262144 is rejected at once); larger
 * batches return WSIM_ESIZE before any metric work.  The first call on a device
 * looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture.  All calls share
 * the array and it keeps the previous call's contents, so calls that overlap
 * on the GPU (other streams, other threads) race: serialise them.  The call
 * synchronises `stream` and returns WSIM_OK or the first error found.  The
 * CSR offsets are device arrays: a first kernel checks them (agent_off and
 * rg_off start at 0, end at N_tot and R_tot and never decrease; at most
 * WSIM_MAX_AGENTS agents per scene) and the call returns WSIM_EINVAL
 * (WSIM_ESIZE for the agent limit) before any kernel reads a scene's
 * roadgraph range; packed segments beyond the limit return WSIM_ESIZE before
 * any is written.  No metric is written on an error.  Outputs are the same
 * as wsim_metrics on the same inputs. */
int wsim_metrics_static(const wsim_config *cfg, const wsim_batch *b, const wsim_state *st,
                        const wsim_metric_buf *m, int t, void *stream);

#ifdef __cplusplus
}
#endif
#endif
