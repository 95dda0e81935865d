/*
 * FP64 CPU oracle for the batched closed-loop driving-simulator step
 * (Waymax, arXiv 2310.08710).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library behind include/wsim.h) never calls it, shares no source with it
 * and has no CPU fallback through it.
 *
 * Every quantity is IEEE double.  Inputs arrive as doubles that the caller
 * up-casts from the same float32 arrays the GPU path reads, so both sides see
 * identical inputs.  Functions are plain definitions by brute force (all pairs,
 * all road-edge segments); the one heuristic (IDM route following) follows its
 * steps in order.  Citations name the paper's section, equation or table.
 *
 * Pins: every function here is checked in tests/test_oracle_*.py against
 * closed forms, brute force or invariants that do not reuse this code
 * (analytic straight-line and constant-curvature trajectories, Sutherland-
 * Hodgman clipping, dense point sampling of polylines, textbook IDM
 * equilibria, central finite differences).
 */
#ifndef WSIM_ORACLE_H
#define WSIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Method constants (the caller passes the same numbers to the GPU path). */
typedef struct {
    double dt;          /* step length, 0.1 s (Sec. 3.1 read as 10 Hz)          */
    double idm_amax;    /* IDM maximum acceleration a (m/s^2)                   */
    double idm_b;       /* IDM comfortable deceleration b (m/s^2)               */
    double idm_T;       /* IDM time headway T (s)                               */
    double idm_s0;      /* IDM minimum gap s0 (m)                               */
    double idm_dq;      /* spacing of the lead-search samples along the route   */
    double route_h;     /* parameter length of one route segment (m)            */
    double gap_min;     /* lower clamp of the bumper gap (m)                    */
    double band;        /* ambiguity band for discrete decisions (m)            */
    int32_t idm_K;      /* number of lead-search samples                        */
    int32_t pad_;
    double kin_amax;    /* kinematic infeasibility: |a| limit, 6 m/s^2 (Sec. 3.4) */
    double kin_kmax;    /* ... |kappa| limit, 0.3 1/m (Sec. 3.4)                 */
    double kin_band_a;  /* band around the |a| limit (m/s^2)                     */
    double kin_band_th; /* band around the turn limit kin_kmax * distance (rad)  */
    double route_max_dist; /* off-route: farther than this from every on-route path (m) */
    double route_max_rel;  /* off-route: an off-route path closer by more than this (m)  */
    /* Discrete action spaces (Sec. 5.2): uniform grids [-max, max] of n values
     * per component.  Bicycle (a, kappa); delta (dx, dy share max/n, dtheta). */
    double disc_a_max, disc_k_max, disc_d_max, disc_t_max;
    int32_t disc_na, disc_nk, disc_nd, disc_nt;
} ob_params;

/* A batch of scenes in CSR form.  Scene s owns agents [agent_off[s],
 * agent_off[s+1]) and roadgraph points [rg_off[s], rg_off[s+1]).  Agent g
 * owns route points [route_off[g], route_off[g+1]) (empty for policy agents).
 * Logs are time-major: log_x[t * N_tot + g]. */
typedef struct {
    int32_t S, N_tot, T_log, pad_;
    const int32_t *agent_off;          /* [S+1]  */
    const int32_t *rg_off;             /* [S+1]  */
    const double  *L, *W, *idm_v0;     /* [N_tot] */
    const uint8_t *valid, *kind;       /* [N_tot] kind: 0 bicycle, 1 delta, 2 IDM */
    const int32_t *route_off;          /* [N_tot+1] */
    const double  *route_x, *route_y;  /* [route_off[N_tot]] */
    const double  *rg_x, *rg_y;        /* [R_tot] */
    const int32_t *rg_poly;            /* [R_tot] polyline id */
    const uint8_t *rg_type, *rg_valid; /* [R_tot] type 1 = road edge */
    const double  *log_x, *log_y;      /* [T_log][N_tot] */
    const double  *log_th, *log_vx, *log_vy; /* [T_log][N_tot]; may be NULL (no expert
                                                or log playback then) */
    /* Route paths of each scene's first agent (may be NULL: no paths): scene
     * s owns paths [path_off[s], path_off[s+1]), path p owns points
     * [path_pt_off[p], path_pt_off[p+1]) in order; path_on[p] = 1 marks an
     * on-route path. */
    const int32_t *path_off, *path_pt_off;
    const double  *path_x, *path_y;
    const uint8_t *path_on;
} ob_batch;

/* Dynamic state per agent, [N_tot] each.  s is the IDM route cursor. */
typedef struct { double *x, *y, *th, *vx, *vy, *s; } ob_state;

/* Per-step metrics, [N_tot] each (reward [S]).
 * flags: bit0 collision, bit1 off-road, bit2 overlap band, bit3 off-road
 * band, bit4 kinematically infeasible transition, bit5 kinematic band (a
 * band bit means the boolean is not gated in parity), bits 6.. reserved. */
typedef struct {
    double  *ov, *off, *logdiv;
    uint8_t *flags;
    int32_t *reward;
} ob_metrics;

/* Who drives an agent (ctrl[g]).  NULL ctrl means OB_CTRL_ACTION for all. */
#define OB_CTRL_HOLD 0    /* keep the state                                       */
#define OB_CTRL_ACTION 1  /* policy agent: the given action                        */
#define OB_CTRL_EXPERT 2  /* policy agent: the expert action fitted to log row t+1 */
#define OB_CTRL_LOG 3     /* any agent: log playback (state := log row t+1)         */
#define OB_CTRL_EXPERT_DISCRETE 4 /* policy agent: the expert action snapped to the
                                     discrete grid (Sec. 5.2)                    */

/* One transition t -> t+1 for scenes [s0, s1) (Sec. 4 step(): all actions are
 * resolved from state t, then every agent moves) into log time index t+1 =
 * t_next (used by the expert and log playback only).  act is [3][N_tot]:
 * (a, kappa, -) for bicycle agents, (dx, dy, dtheta) for delta agents;
 * IDM agents ignore it and follow their route unless ctrl = OB_CTRL_LOG.
 * Invalid agents keep their state.  band_idm[g] (may be NULL) is set to 1
 * when an IDM decision of agent g lies inside the ambiguity band; lead[g]
 * (may be NULL) receives the chosen lead agent (global index) or -1. */
int oracle_transition(const ob_params *p, const ob_batch *b, int s0, int s1,
                      const ob_state *in, const double *act, const uint8_t *ctrl, int t_next,
                      ob_state *out, uint8_t *band_idm, int32_t *lead);

/* Metrics of state st at time index t (log row t) for scenes [s0, s1):
 * overlap (Sec. 3.4 collision), off-road (Sec. 3.4), log divergence
 * (Sec. 3.4 displacement error), the sparse reward (Sec. 5.2) and, when prev
 * (the state at t-1) is given, kinematic infeasibility of the transition
 * prev -> st (Sec. 3.4). */
int oracle_metrics(const ob_params *p, const ob_batch *b, int s0, int s1,
                   const ob_state *st, const ob_state *prev, int t, ob_metrics *m);

/* Free-running rollout of T steps from time index t0 for scenes [s0, s1):
 * st holds state t0 on entry and state t0+T on exit; act_seq is
 * [T][3][N_tot] (may be NULL when no agent takes OB_CTRL_ACTION); ctrl as in
 * oracle_transition (may be NULL); metric arrays are [T][N_tot] (reward
 * [T][S]).  Scenes are split over nthreads OpenMP threads (<= 0: all cores). */
int oracle_rollout(const ob_params *p, const ob_batch *b, int s0, int s1,
                   ob_state *st, const double *act_seq, const uint8_t *ctrl, int t0, int T,
                   ob_metrics *mseq, int nthreads);

/* Discrete actions (Sec. 5.2: a discrete action space's inverse is the
 * continuous inverse, discretised).  The index of a value v on a grid of n
 * values over [-max, max] is rint(fl(fl(v) / step) + c) clamped to [0, n-1],
 * with step = fl(2 max / (n-1)) and c = (n-1)/2, in float32 (an integer
 * decision taken in the kernel's precision); the grid value of index i is
 * fl(fl(i - c) * step), so an odd n puts 0 on the grid.  Flat index:
 * bicycle i_a * n_k + i_k; delta (i_x * n_d + i_y) * n_t + i_t.
 * oracle_discretize: act [T][3][N_tot] -> idx [T][N_tot] (-1 for IDM and
 * invalid agents); band[T][N_tot] (may be NULL) = 1 when some component's
 * scaled value lies within 1e-3 of a rounding boundary.
 * oracle_decode_actions: idx -> act (grid values; 0 for idx < 0). */
int oracle_discretize(const ob_params *p, const ob_batch *b, const double *act, int T, int32_t *idx,
                      uint8_t *band);
int oracle_decode_actions(const ob_params *p, const ob_batch *b, const int32_t *idx, int T, double *act);

/* Inverse of the action spaces (App. A.1) for every agent of scenes [s0, s1):
 * the action that takes state prev to state next, written to act [3][N_tot]:
 * bicycle agents (a, kappa, 0) by the inverse kinematics, delta agents
 * (x'-x, y'-y, theta'-theta); IDM and invalid agents 0. */
int oracle_inverse(const ob_params *p, const ob_batch *b, int s0, int s1,
                   const ob_state *prev, const ob_state *next, double *act);

/* Expert actions (Sec. 5.2, open loop): act_seq[k] = the inverse of log row
 * t0+k -> log row t0+k+1 for k < T, [T][3][N_tot], as oracle_inverse. */
int oracle_expert_actions(const ob_params *p, const ob_batch *b, int s0, int s1,
                          int t0, int T, double *act_seq);

/* Observation (Sec. 3.2: other agents in the agent's own frame, the
 * roadgraph subsampled by distance) of state st for every agent g of scenes
 * [s0, s1) with observers[g] != 0 (observers NULL: every valid agent).  The
 * frame of g: origin at g's centre, x axis along its heading.
 * agents[(g*M + j)*5 + c], c = x, y, yaw, vx, vy: agent j (index within g's
 * scene) in g's frame, yaw reduced to [-pi, pi]; agents_valid[g*M + j] = 1
 * iff agent j is valid and j != g (other entries 0).  rg[(g*K + k)*2 + c]
 * and rg_idx[g*K + k]: the K valid roadgraph points (any type) of g's scene
 * nearest to g's centre, ascending, ties to the lower global point index,
 * in g's frame; -1 and 0 past the scene's valid points.  Reading: the
 * ranking key is float32 (the precision of the GPU kernel, which makes the
 * same integer decision): c = float(centre), d = float(p - c), key =
 * fmaf(dx, dx, dy*dy).  Rows of non-observers are not written.  Requires
 * M >= agents of every scene in range, K >= 1. */
int oracle_observe(const ob_params *p, const ob_batch *b, int s0, int s1, const ob_state *st,
                   const uint8_t *observers, int M, int K, double *agents, uint8_t *agents_valid,
                   double *rg, int32_t *rg_idx);

/* Route metrics (Sec. 3.4) of the first agent of each scene in [s0, s1) at
 * state st: progress[s] = (d_x - d_p) / (d_q - d_p), where d_x is the arc
 * length along the on-route path nearest to the agent (ties: lower path) of
 * the agent's nearest point on it (ties: lower segment), and d_p, d_q those
 * of the first and last logged positions (log rows 0 and T_log-1) on the
 * same path; NaN when d_q - d_p <= 1e-3 m or the scene has no on-route
 * path.  flags[s]: bit0 off-route (distance to the nearest on-route path >
 * route_max_dist, or an off-route path nearer by more than route_max_rel),
 * bit1 band (a deciding distance within p->band of its threshold), bit2
 * progress ambiguous (two on-route paths, or two non-adjacent segments of
 * the chosen path, within p->band of the nearest). */
int oracle_route(const ob_params *p, const ob_batch *b, int s0, int s1, const ob_state *st,
                 double *progress, uint8_t *flags);

/* Signed SAT depth of two boxes (centre, heading, length, width):
 * > 0 iff the boxes overlap (then it is the minimum translation distance). */
double oracle_box_depth(const double *box_a, const double *box_b);

/* Signed distance of point (px, py) to the road edges of scene s (> 0 means
 * off road); *ambiguous is set when a near tie between non-adjacent
 * segments of opposite sign lies inside the band.  Returns -inf when the
 * scene has no road-edge segment; *seg_out (may be NULL) receives the global
 * roadgraph index of the winning segment's start point, or -1. */
double oracle_point_sd(const ob_params *p, const ob_batch *b, int s,
                       double px, double py, int *ambiguous, int32_t *seg_out);

/* Differentiable loss of one scene over T steps:
 * L = sum_t sum_i d_i(t)^2 + lambda * sum_t sum_{i<j} tau*softplus(d_ij/tau)
 * over valid agents.  IDM agents move as in oracle_transition but are
 * constants for differentiation (stop-gradient). */
double oracle_loss(const ob_params *p, const ob_batch *b, int s,
                   const ob_state *st0, const double *act_seq, int t0, int T,
                   double lambda, double tau);

/* dL/d act_seq[t][c][g] for n directions by forward-mode dual numbers
 * (one pass per direction), written to grad[n]. */
int oracle_loss_grad(const ob_params *p, const ob_batch *b, int s,
                     const ob_state *st0, const double *act_seq, int t0, int T,
                     double lambda, double tau, int n, const int32_t *dir_t,
                     const int32_t *dir_c, const int32_t *dir_g, double *grad);

/* Differentiable objective of one scene over T steps (the objective whose
 * gradient the differentiable rollout returns):
 *   J = w_loss * L + sum_k sum_g ( g_logdiv[k][g] * d_g(t0+k+1)
 *                                + g_ov[k][g] * ov_g(t0+k+1) + g_off[k][g] * off_g(t0+k+1) )
 * with L the loss of oracle_loss and d, ov, off the metrics of oracle_metrics
 * (log divergence, largest SAT depth against another valid agent, largest
 * signed distance of a box corner to the road edges) of the rollout's states.
 * Weight arrays are [T][N_tot] (element k * N_tot + g), each may be NULL
 * (all 0); a metric of weight 0 is not evaluated and a metric of -inf adds
 * nothing.  The max over partners and corners keeps the first maximum
 * (lowest partner index, corner order of oracle_metrics); the nearest road
 * edge and its side are decided on the values.  IDM agents move but are
 * constants for differentiation. */
double oracle_objective(const ob_params *p, const ob_batch *b, int s, const ob_state *st0,
                        const double *act_seq, int t0, int T, double lambda, double tau, double w_loss,
                        const double *g_logdiv, const double *g_ov, const double *g_off);

/* dJ/d(direction) for n directions by forward-mode dual numbers (one pass
 * each): dir_kind 0 = act_seq[dir_t][dir_c][dir_g] (dir_c 0..2); dir_kind 1 =
 * component dir_c (0 x, 1 y, 2 theta, 3 vx, 4 vy) of agent dir_g's initial
 * state (dir_t unused).  Returns 0, or -1 for a bad direction or a scene
 * that cannot be rolled out. */
int oracle_objective_grad(const ob_params *p, const ob_batch *b, int s, const ob_state *st0,
                          const double *act_seq, int t0, int T, double lambda, double tau, double w_loss,
                          const double *g_logdiv, const double *g_ov, const double *g_off, int n,
                          const int32_t *dir_kind, const int32_t *dir_t, const int32_t *dir_c,
                          const int32_t *dir_g, double *grad);

#ifdef __cplusplus
}
#endif
#endif
