// FP64 CPU oracle for the batched closed-loop driving-simulator step
// (Waymax, arXiv 2310.08710).  TEST INFRASTRUCTURE ONLY: see oracle.h.
//
// Plain definitions by brute force: every agent pair, every road-edge segment,
// one dual-number pass per gradient direction.  Nothing is blocked, culled or
// reordered beyond what the definitions state, so each function can be checked
// against the paper by eye.  Readings of points the paper leaves open are
// marked "Reading:" and repeated in the design notes.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kInf = std::numeric_limits<double>::infinity();
const double kTwoPi = 2.0 * std::acos(-1.0);

// ---------------------------------------------------------------------------
// Forward-mode dual numbers (value, one tangent) for the loss gradient.
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double x) : v(x), d(0) {}  // NOLINT: implicit lift of constants
    Dual(double x, double t) : v(x), d(t) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
    return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual sqrt(Dual a) {
    double r = std::sqrt(a.v);
    return {r, r > 0 ? a.d / (2 * r) : 0.0};
}
inline Dual sin(Dual a) { return {std::sin(a.v), std::cos(a.v) * a.d}; }
inline Dual cos(Dual a) { return {std::cos(a.v), -std::sin(a.v) * a.d}; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }
inline Dual log1p(Dual a) { return {std::log1p(a.v), a.d / (1 + a.v)}; }
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
template <class T> inline T tmin(T a, T b) { return val(b) < val(a) ? b : a; }
template <class T> inline T tmax(T a, T b) { return val(b) > val(a) ? b : a; }

using std::cos;
using std::exp;
using std::fabs;
using std::log1p;
using std::sin;
using std::sqrt;

// ---------------------------------------------------------------------------
// Agent state and the two dynamics models of App. A.1.
// ---------------------------------------------------------------------------
template <class T> struct St { T x, y, th, vx, vy; };

// App. A.1, bicycle action space, forward dynamics: position advanced with the
// current velocity plus half the acceleration along the current heading; the
// heading turns by kappa times the distance travelled; the new speed is put
// along the new heading.  Reading: no clamp of v' (the equations have none).
template <class T>
St<T> bicycle_forward(const St<T>& s, T a, T kappa, double dt) {
    T v = sqrt(s.vx * s.vx + s.vy * s.vy);
    St<T> o;
    o.x = s.x + s.vx * dt + 0.5 * a * cos(s.th) * dt * dt;
    o.y = s.y + s.vy * dt + 0.5 * a * sin(s.th) * dt * dt;
    o.th = s.th + kappa * (v * dt + 0.5 * a * dt * dt);
    T vn = v + a * dt;
    o.vx = vn * cos(o.th);
    o.vy = vn * sin(o.th);
    return o;
}

// App. A.1, delta action space: displacements added, velocity is the
// displacement over the step length.
template <class T>
St<T> delta_forward(const St<T>& s, T dx, T dy, T dth, double dt) {
    St<T> o;
    o.x = s.x + dx;
    o.y = s.y + dy;
    o.th = s.th + dth;
    o.vx = (o.x - s.x) / dt;
    o.vy = (o.y - s.y) / dt;
    return o;
}

// App. A.1, inverse kinematics of the bicycle action space, from two
// consecutive states: the acceleration is the change of speed over one step;
// the curvature is the turn of the direction of travel divided by the
// distance travelled, v dt + a dt^2 / 2.  Readings: the direction of the new
// state is the heading of its velocity, atan2(vy', vx') (the paper prints
// arctan(vx'/vy'), which swaps the components and loses the quadrant); the
// turn away from the old heading is reduced modulo 2 pi into [-pi, pi]; a
// state with zero velocity has no direction, so the turn is 0; with no
// distance travelled the curvature is 0.
struct BicycleInverse { double a, kappa, turn, dist; bool has_dir; };

BicycleInverse bicycle_inverse(const St<double>& s, const St<double>& n, double dt) {
    BicycleInverse r;
    const double v = std::sqrt(s.vx * s.vx + s.vy * s.vy);
    const double vn = std::sqrt(n.vx * n.vx + n.vy * n.vy);
    r.a = (vn - v) / dt;
    r.has_dir = n.vx != 0.0 || n.vy != 0.0;
    r.turn = r.has_dir ? std::remainder(std::atan2(n.vy, n.vx) - s.th, kTwoPi) : 0.0;
    r.dist = v * dt + 0.5 * r.a * dt * dt;
    r.kappa = r.dist > 0 ? r.turn / r.dist : 0.0;
    return r;
}

// Sec. 3.4, kinematic infeasibility of the transition s -> n: the inverse
// kinematics estimate breaks |a| <= kin_amax or |kappa| <= kin_kmax.  *band
// is set when either comparison lies inside its band: |a| against the limit,
// or the turn against kin_kmax times the distance (the curvature test with
// the distance multiplied out, which stays defined for short steps).  A new
// state without velocity has no direction and a turn of exactly 0, so its
// curvature decision is exact and never in the band.
void kin_check(const ob_params* p, const St<double>& s, const St<double>& n, bool* flag, bool* band) {
    const BicycleInverse r = bicycle_inverse(s, n, p->dt);
    *flag = std::fabs(r.a) > p->kin_amax || std::fabs(r.kappa) > p->kin_kmax;
    *band = std::fabs(std::fabs(r.a) - p->kin_amax) <= p->kin_band_a ||
            (r.has_dir && std::fabs(std::fabs(r.turn) - p->kin_kmax * r.dist) <= p->kin_band_th);
}

bool has_full_log(const ob_batch* b) { return b->log_th && b->log_vx && b->log_vy; }

// Grid index of v on n values over [-max, max] (float32, see oracle.h);
// *near = the scaled value lies within 1e-3 of a rounding boundary.
int disc_index(double v, double max, int n, bool* near) {
    const float step = 2.0f * (float)max / (float)(n - 1);
    const float c = 0.5f * (float)(n - 1);
    const float q = (float)v / step + c;
    const float r = std::rint(q);
    if (near && std::fabs(std::fabs(q - std::floor(q)) - 0.5f) < 1e-3f && q > -0.5f && q < n - 0.5f) *near = true;
    return (int)std::min((float)(n - 1), std::max(0.0f, r));
}
float disc_value(int i, double max, int n) {
    const float step = 2.0f * (float)max / (float)(n - 1);
    const float c = 0.5f * (float)(n - 1);
    return ((float)i - c) * step;
}

// Flat discrete index of an action of agent kind `kind` (-1 for IDM).
int disc_encode(const ob_params* p, int kind, const double u[3], bool* near) {
    if (kind == 0)
        return disc_index(u[0], p->disc_a_max, p->disc_na, near) * p->disc_nk +
               disc_index(u[1], p->disc_k_max, p->disc_nk, near);
    if (kind == 1)
        return (disc_index(u[0], p->disc_d_max, p->disc_nd, near) * p->disc_nd +
                disc_index(u[1], p->disc_d_max, p->disc_nd, near)) * p->disc_nt +
               disc_index(u[2], p->disc_t_max, p->disc_nt, near);
    return -1;
}
void disc_decode(const ob_params* p, int kind, int idx, double u[3]) {
    u[0] = u[1] = u[2] = 0.0;
    if (idx < 0) return;
    if (kind == 0) {
        u[0] = disc_value(idx / p->disc_nk, p->disc_a_max, p->disc_na);
        u[1] = disc_value(idx % p->disc_nk, p->disc_k_max, p->disc_nk);
    } else if (kind == 1) {
        const int it = idx % p->disc_nt, ixy = idx / p->disc_nt;
        u[0] = disc_value(ixy / p->disc_nd, p->disc_d_max, p->disc_nd);
        u[1] = disc_value(ixy % p->disc_nd, p->disc_d_max, p->disc_nd);
        u[2] = disc_value(it, p->disc_t_max, p->disc_nt);
    }
}

St<double> log_state(const ob_batch* b, int t, int g) {
    const size_t i = (size_t)t * b->N_tot + g;
    return {b->log_x[i], b->log_y[i], b->log_th[i], b->log_vx[i], b->log_vy[i]};
}

St<double> get_state(const ob_state* st, int g) { return {st->x[g], st->y[g], st->th[g], st->vx[g], st->vy[g]}; }

// The action of agent g's action space that takes state s to state n (App.
// A.1 inverses): bicycle (a, kappa, 0), delta (x'-x, y'-y, theta'-theta).
void inverse_action(const ob_params* p, int kind, const St<double>& s, const St<double>& n, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (kind == 0) {
        const BicycleInverse r = bicycle_inverse(s, n, p->dt);
        out[0] = r.a;
        out[1] = r.kappa;
    } else if (kind == 1) {
        out[0] = n.x - s.x;
        out[1] = n.y - s.y;
        out[2] = n.th - s.th;
    }
}

// ---------------------------------------------------------------------------
// Oriented boxes and the separating-axis overlap depth (Sec. 3.4, collision:
// two top-down boxes at the same step overlap).
// ---------------------------------------------------------------------------
template <class T> struct Box { T cx, cy, c, s, hl, hw; };

template <class T> Box<T> make_box(T x, T y, T th, double L, double W) {
    Box<T> b;
    b.cx = x; b.cy = y; b.c = cos(th); b.s = sin(th);
    b.hl = T(0.5 * L); b.hw = T(0.5 * W);
    return b;
}

// Signed depth d = min over the four edge normals of (rA + rB - |dc . axis|),
// rX being box X's half extent projected on the axis.  d > 0 iff the boxes
// overlap (no separating axis among the edge normals of two rectangles); then
// d is the minimum translation distance.
template <class T> T sat_depth(const Box<T>& A, const Box<T>& B) {
    T dx = B.cx - A.cx, dy = B.cy - A.cy;
    T ax[4] = {A.c, -A.s, B.c, -B.s};
    T ay[4] = {A.s, A.c, B.s, B.c};
    T best = T(kInf);
    for (int k = 0; k < 4; ++k) {
        T rA = A.hl * fabs(A.c * ax[k] + A.s * ay[k]) + A.hw * fabs(-A.s * ax[k] + A.c * ay[k]);
        T rB = B.hl * fabs(B.c * ax[k] + B.s * ay[k]) + B.hw * fabs(-B.s * ax[k] + B.c * ay[k]);
        T ov = rA + rB - fabs(dx * ax[k] + dy * ay[k]);
        best = tmin(best, ov);
    }
    return best;
}

// Numerically stable softplus: max(x,0) + log(1 + exp(-|x|)).
template <class T> T softplus(T x) { return tmax(x, T(0.0)) + log1p(exp(-fabs(x))); }

// ---------------------------------------------------------------------------
// Road-edge segments (Sec. 3.4 off-road: the vehicle must be on the left of the
// oriented road edge).  Points k and k+1 form a segment iff both are valid road
// edges of the same polyline; it is oriented k -> k+1.
// ---------------------------------------------------------------------------
struct Seg { double ax, ay, ux, uy; int k; int prev, next; };

bool is_seg(const ob_batch* b, int r0, int r1, int k) {
    if (k < r0 || k + 1 >= r1) return false;
    return b->rg_valid[k] && b->rg_valid[k + 1] && b->rg_type[k] == 1 &&
           b->rg_type[k + 1] == 1 && b->rg_poly[k] == b->rg_poly[k + 1];
}

std::vector<Seg> scene_segments(const ob_batch* b, int s) {
    int r0 = b->rg_off[s], r1 = b->rg_off[s + 1];
    std::vector<Seg> v;
    for (int k = r0; k + 1 < r1; ++k) {
        if (!is_seg(b, r0, r1, k)) continue;
        Seg g;
        g.ax = b->rg_x[k]; g.ay = b->rg_y[k];
        g.ux = b->rg_x[k + 1] - b->rg_x[k];
        g.uy = b->rg_y[k + 1] - b->rg_y[k];
        g.k = k;
        g.prev = is_seg(b, r0, r1, k - 1) ? (int)v.size() - 1 : -1;
        g.next = -1;
        if (g.prev >= 0) v[g.prev].next = (int)v.size();
        v.push_back(g);
    }
    return v;
}

inline double cross(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

// Which side of the nearest feature point p lies on: true = left = on road.
// Interior nearest point (or an open polyline end): sign of u x (p - a).
// Reading (the paper is silent on vertices): at a shared vertex with incoming
// u1 and outgoing u2, a left turn (u1 x u2 > 0) keeps p on road iff it is left
// of both lines, a right turn iff it is left of either, collinear uses u1.
bool on_road_side(const std::vector<Seg>& g, int i, double traw, double px, double py) {
    const Seg& e = g[i];
    double vx, vy, u1x, u1y, u2x, u2y;
    if (traw <= 0 && e.prev >= 0) {
        vx = e.ax; vy = e.ay;
        u1x = g[e.prev].ux; u1y = g[e.prev].uy; u2x = e.ux; u2y = e.uy;
    } else if (traw >= 1 && e.next >= 0) {
        vx = e.ax + e.ux; vy = e.ay + e.uy;
        u1x = e.ux; u1y = e.uy; u2x = g[e.next].ux; u2y = g[e.next].uy;
    } else {
        return cross(e.ux, e.uy, px - e.ax, py - e.ay) > 0;
    }
    bool l1 = cross(u1x, u1y, px - vx, py - vy) > 0;
    bool l2 = cross(u2x, u2y, px - vx, py - vy) > 0;
    double turn = cross(u1x, u1y, u2x, u2y);
    if (turn > 0) return l1 && l2;
    if (turn < 0) return l1 || l2;
    return l1;
}

// Distance of p to segment i; traw is the unclamped projection parameter.
inline double seg_d2(const Seg& e, double px, double py, double* traw) {
    double wx = px - e.ax, wy = py - e.ay;
    double t = (wx * e.ux + wy * e.uy) / (e.ux * e.ux + e.uy * e.uy);
    *traw = t;
    double tc = std::min(1.0, std::max(0.0, t));
    double ex = wx - tc * e.ux, ey = wy - tc * e.uy;
    return ex * ex + ey * ey;
}

// Exhaustive nearest-segment scan (ties go to the lower roadgraph index) and
// the signed distance: -dist on road, +dist off road.
double point_sd(const std::vector<Seg>& g, double px, double py, double band,
                int* ambiguous, int* seg_index) {
    int best = -1;
    double bd2 = kInf, bt = 0;
    for (int i = 0; i < (int)g.size(); ++i) {
        double t, d2 = seg_d2(g[i], px, py, &t);
        if (d2 < bd2) { bd2 = d2; best = i; bt = t; }
    }
    if (seg_index) *seg_index = best;
    if (best < 0) { if (ambiguous) *ambiguous = 0; return -kInf; }
    bool on = on_road_side(g, best, bt, px, py);
    double bd = std::sqrt(bd2);
    if (ambiguous) {
        // A near tie with a segment that shares no vertex with the winner and
        // puts p on the other side: the sign is not decided robustly.
        *ambiguous = 0;
        for (int i = 0; i < (int)g.size(); ++i) {
            if (i == best || i == g[best].prev || i == g[best].next) continue;
            double t, d2 = seg_d2(g[i], px, py, &t);
            if (std::sqrt(d2) > bd + band) continue;
            if (on_road_side(g, i, t, px, py) != on) { *ambiguous = 1; break; }
        }
    }
    return on ? -bd : bd;
}

// ---------------------------------------------------------------------------
// IDM route following (Sec. 3.5: follow the logged path, IDM sets the speed).
// The paper gives no equations; this is the textbook IDM of Treiber et al.
// (2000), which the paper cites, with a lead search along the route.
// ---------------------------------------------------------------------------
struct RoutePt { double x, y, tx, ty; int seg; };

// Position on the route polyline at parameter s: segment k = floor(s/h)
// (clamped to the route, the last segment extrapolated), linear inside it.
RoutePt route_eval(const double* rx, const double* ry, int P, double h, double s) {
    double u = s / h;
    int k = (int)std::floor(u);
    if (k < 0) k = 0;
    if (k > P - 2) k = P - 2;
    double tau = u - k;
    double dx = rx[k + 1] - rx[k], dy = ry[k + 1] - ry[k];
    double n = std::sqrt(dx * dx + dy * dy);
    RoutePt r;
    r.x = rx[k] + tau * dx;
    r.y = ry[k] + tau * dy;
    r.tx = dx / n; r.ty = dy / n;
    r.seg = k;
    return r;
}

// True when s lies within eps (metres) of the boundary between two route
// segments of different heading: the segment (hence heading) chosen at s is
// then not decided robustly.
bool boundary_ambiguous(const double* rx, const double* ry, int P, double h, double s, double eps) {
    double u = s / h;
    double j = std::nearbyint(u);
    if (std::fabs(u - j) * h >= eps) return false;
    int k = (int)j;
    if (k <= 0 || k >= P - 1) return false;  // both sides clamp to the same segment
    double ax = rx[k] - rx[k - 1], ay = ry[k] - ry[k - 1];
    double bx = rx[k + 1] - rx[k], by = ry[k + 1] - ry[k];
    return std::fabs(cross(ax, ay, bx, by)) > 1e-12 * (ax * ax + ay * ay);
}

struct IdmOut { St<double> st; double s; int lead; bool band; };

// The agent state arrays of `in` are indexed by (global agent index - base).
IdmOut idm_agent(const ob_params* p, const ob_batch* b, int a0, int a1, int i,
                 const ob_state* in, int base = 0) {
    const double h = p->route_h, eps = p->band;
    const int ro = b->route_off[i], P = b->route_off[i + 1] - ro;
    const double* rx = b->route_x + ro;
    const double* ry = b->route_y + ro;
    const double xi = in->x[i - base], yi = in->y[i - base], si = in->s[i - base];
    const double v = std::sqrt(in->vx[i - base] * in->vx[i - base] + in->vy[i - base] * in->vy[i - base]);
    const double Li = b->L[i], Wi = b->W[i];
    const int K = p->idm_K;
    bool band = false;

    // Lead-search samples ahead of the front bumper along the route.
    std::vector<RoutePt> q(K + 1);
    for (int k = 1; k <= K; ++k) q[k] = route_eval(rx, ry, P, h, si + 0.5 * Li + p->idm_dq * k);

    // Candidates: another valid agent whose box, widened by half this agent's
    // width, contains a sample.  first_hit = first such sample.
    int lead = -1, lead_hit = -1;
    double g1 = kInf, g2 = kInf, raw1 = kInf, raw2 = kInf;
    std::vector<double> nonrobust_gaps;
    for (int j = a0; j < a1; ++j) {
        if (j == i || !b->valid[j]) continue;
        double cj = std::cos(in->th[j - base]), sj = std::sin(in->th[j - base]);
        int first = -1;
        bool firm = false, maybe = false;
        for (int k = 1; k <= K; ++k) {
            double rxq = q[k].x - in->x[j - base], ryq = q[k].y - in->y[j - base];
            double pu = std::fabs(rxq * cj + ryq * sj);
            double pn = std::fabs(-rxq * sj + ryq * cj);
            double m = std::min(0.5 * b->L[j] + 0.5 * Wi - pu, 0.5 * b->W[j] + 0.5 * Wi - pn);
            if (m >= 0 && first < 0) first = k;
            if (m >= eps) firm = true;
            if (std::fabs(m) < eps) maybe = true;
        }
        double dist = std::sqrt((in->x[j - base] - xi) * (in->x[j - base] - xi) + (in->y[j - base] - yi) * (in->y[j - base] - yi));
        double raw = dist - 0.5 * (Li + b->L[j]);
        double g = std::max(p->gap_min, raw);
        if (maybe && !firm) nonrobust_gaps.push_back(g);
        if (first < 0) continue;
        if (g < g1) {
            g2 = g1; raw2 = raw1; g1 = g; raw1 = raw; lead = j; lead_hit = first;
        } else if (g < g2) {
            g2 = g; raw2 = raw;
        }
    }
    // Ambiguity band: a candidate that a float32 test could add or drop and
    // that could win; a near tie of the two smallest gaps (unless both sit on
    // the clamp); an uncertain first-hit sample of the lead.
    for (double g : nonrobust_gaps)
        if (lead < 0 || g <= g1 + eps) band = true;
    if (lead >= 0 && g2 - g1 < eps && !(raw1 < p->gap_min - eps && raw2 < p->gap_min - eps))
        band = true;
    double vlead = 0;
    if (lead >= 0) {
        double cj = std::cos(in->th[lead - base]), sj = std::sin(in->th[lead - base]);
        for (int k = 1; k <= lead_hit; ++k) {
            double rxq = q[k].x - in->x[lead - base], ryq = q[k].y - in->y[lead - base];
            double pu = std::fabs(rxq * cj + ryq * sj);
            double pn = std::fabs(-rxq * sj + ryq * cj);
            double m = std::min(0.5 * b->L[lead] + 0.5 * Wi - pu, 0.5 * b->W[lead] + 0.5 * Wi - pn);
            if (std::fabs(m) < eps) band = true;
        }
        if (boundary_ambiguous(rx, ry, P, h, si + 0.5 * Li + p->idm_dq * lead_hit, eps)) band = true;
        vlead = in->vx[lead - base] * q[lead_hit].tx + in->vy[lead - base] * q[lead_hit].ty;
    }

    // Textbook IDM acceleration (delta = 4).
    const double v0 = b->idm_v0[i];
    double r4 = (v / v0) * (v / v0) * (v / v0) * (v / v0);
    double acc;
    if (lead >= 0) {
        double dv = v - vlead;
        double sstar = p->idm_s0 + std::max(0.0, v * p->idm_T + v * dv / (2 * std::sqrt(p->idm_amax * p->idm_b)));
        acc = p->idm_amax * (1 - r4 - (sstar / g1) * (sstar / g1));
    } else {
        acc = p->idm_amax * (1 - r4);
    }
    // Advance along the route with the trapezoidal distance of the new speed.
    double vn = std::max(0.0, v + acc * p->dt);
    double sn = si + 0.5 * (v + vn) * p->dt;
    RoutePt r = route_eval(rx, ry, P, h, sn);
    if (boundary_ambiguous(rx, ry, P, h, sn, eps)) band = true;
    IdmOut o;
    o.st.x = r.x; o.st.y = r.y;
    o.st.th = std::atan2(r.ty, r.tx);
    o.st.vx = vn * std::cos(o.st.th);
    o.st.vy = vn * std::sin(o.st.th);
    o.s = sn;
    o.lead = lead;
    o.band = band;
    return o;
}

void copy_agent(const ob_state* in, ob_state* out, int g) {
    out->x[g] = in->x[g]; out->y[g] = in->y[g]; out->th[g] = in->th[g];
    out->vx[g] = in->vx[g]; out->vy[g] = in->vy[g]; out->s[g] = in->s[g];
}

void put_state(ob_state* out, int g, const St<double>& n) {
    out->x[g] = n.x; out->y[g] = n.y; out->th[g] = n.th; out->vx[g] = n.vx; out->vy[g] = n.vy;
}

int transition_scene(const ob_params* p, const ob_batch* b, int s, const ob_state* in,
                     const double* act, const uint8_t* ctrl, int t_next, ob_state* out,
                     uint8_t* band_idm, int32_t* lead_out) {
    const int a0 = b->agent_off[s], a1 = b->agent_off[s + 1], N = b->N_tot;
    for (int g = a0; g < a1; ++g) {
        if (band_idm) band_idm[g] = 0;
        if (lead_out) lead_out[g] = -1;
        const int kind = b->kind[g];
        const int cm = ctrl ? ctrl[g] : OB_CTRL_ACTION;
        if (cm > OB_CTRL_EXPERT_DISCRETE) return -1;
        if (!b->valid[g] || (kind != 2 && cm == OB_CTRL_HOLD)) { copy_agent(in, out, g); continue; }
        const bool expert = cm == OB_CTRL_EXPERT || cm == OB_CTRL_EXPERT_DISCRETE;
        const bool needs_log = cm == OB_CTRL_LOG || (expert && kind != 2);
        if (needs_log && (!has_full_log(b) || t_next < 0 || t_next >= b->T_log)) return -1;
        if (cm == OB_CTRL_LOG) {  // log playback (Sec. 3.5): the logged state of t+1
            put_state(out, g, log_state(b, t_next, g));
            out->s[g] = in->s[g];
            continue;
        }
        if (kind != 2 && cm == OB_CTRL_ACTION && !act) return -1;
        St<double> cur = get_state(in, g);
        if (kind == 0 || kind == 1) {
            double u[3];
            if (expert) {  // Sec. 5.2 expert: the action fitted to the log
                inverse_action(p, kind, cur, log_state(b, t_next, g), u);
                if (cm == OB_CTRL_EXPERT_DISCRETE) {  // ... snapped to the discrete grid
                    bool near = false;
                    const int idx = disc_encode(p, kind, u, &near);
                    disc_decode(p, kind, idx, u);
                    if (band_idm && near) band_idm[g] = 1;
                }
            } else {
                u[0] = act[g]; u[1] = act[N + g]; u[2] = act[2 * N + g];
            }
            St<double> n = kind == 0 ? bicycle_forward(cur, u[0], u[1], p->dt)
                                     : delta_forward(cur, u[0], u[1], u[2], p->dt);
            put_state(out, g, n);
            out->s[g] = in->s[g];
        } else if (kind == 2) {
            if (b->route_off[g + 1] - b->route_off[g] < 2) return -1;
            IdmOut o = idm_agent(p, b, a0, a1, g, in);
            out->x[g] = o.st.x; out->y[g] = o.st.y; out->th[g] = o.st.th;
            out->vx[g] = o.st.vx; out->vy[g] = o.st.vy; out->s[g] = o.s;
            if (band_idm) band_idm[g] = o.band;
            if (lead_out) lead_out[g] = o.lead;
        } else {
            return -1;
        }
    }
    return 0;
}

// Metrics of one scene (Sec. 3.4) on state st, log row t; prev (may be NULL)
// is the state before, for kinematic infeasibility.
void metrics_scene(const ob_params* p, const ob_batch* b, int s, const ob_state* st, const ob_state* prev,
                   int t, double* ov, double* off, double* logdiv, uint8_t* flags, int32_t* reward) {
    const int a0 = b->agent_off[s], a1 = b->agent_off[s + 1], N = b->N_tot;
    const double eps = p->band;
    std::vector<Box<double>> box(a1 - a0);
    for (int g = a0; g < a1; ++g) box[g - a0] = make_box(st->x[g], st->y[g], st->th[g], b->L[g], b->W[g]);
    std::vector<Seg> segs = scene_segments(b, s);
    int32_t r = 0;
    for (int g = a0; g < a1; ++g) {
        if (!b->valid[g]) { ov[g] = off[g] = logdiv[g] = 0; flags[g] = 0; continue; }
        // Collision: largest SAT depth against any other valid agent.
        double o = -kInf;
        for (int j = a0; j < a1; ++j) {
            if (j == g || !b->valid[j]) continue;
            int lo = std::min(g, j), hi = std::max(g, j);
            o = std::max(o, sat_depth(box[lo - a0], box[hi - a0]));
        }
        // Off-road: largest signed distance over the four box corners.
        const Box<double>& B = box[g - a0];
        double f = -kInf;
        int amb_any = 0;
        const double sl[4] = {1, 1, -1, -1}, sw[4] = {1, -1, -1, 1};
        for (int c = 0; c < 4; ++c) {
            double px = B.cx + sl[c] * B.hl * B.c - sw[c] * B.hw * B.s;
            double py = B.cy + sl[c] * B.hl * B.s + sw[c] * B.hw * B.c;
            int amb = 0;
            f = std::max(f, point_sd(segs, px, py, eps, &amb, nullptr));
            amb_any |= amb;
        }
        // Log divergence: L2 distance to the logged position at the same step.
        double dx = st->x[g] - b->log_x[(size_t)t * N + g];
        double dy = st->y[g] - b->log_y[(size_t)t * N + g];
        ov[g] = o;
        off[g] = f;
        logdiv[g] = std::sqrt(dx * dx + dy * dy);
        uint8_t fl = 0;
        if (o > 0) fl |= 1;
        if (f > 0) fl |= 2;
        if (std::fabs(o) < eps) fl |= 4;
        if (std::fabs(f) < eps || amb_any) fl |= 8;
        if (prev) {
            bool kf = false, kb = false;
            kin_check(p, get_state(prev, g), get_state(st, g), &kf, &kb);
            if (kf) fl |= 16;
            if (kb) fl |= 32;
        }
        flags[g] = fl;
        r -= (o > 0) + (f > 0);
    }
    reward[s] = r;
}

// Signed distance of a point whose coordinates may carry derivatives
// (Sec. 3.4 off-road).  The nearest segment and the side are decided on the
// values, exactly as point_sd decides them (exhaustive scan, ties to the
// lower index, vertex rule); the distance from the point to that segment's
// nearest point (the projection parameter clamped to [0, 1]) carries the
// derivative.
template <class T> T point_sd_t(const std::vector<Seg>& g, T px, T py) {
    int idx = -1;
    point_sd(g, val(px), val(py), 0.0, nullptr, &idx);
    if (idx < 0) return T(-kInf);
    const Seg& e = g[idx];
    double traw;
    seg_d2(e, val(px), val(py), &traw);
    const bool on = on_road_side(g, idx, traw, val(px), val(py));
    T wx = px - e.ax, wy = py - e.ay;
    T t = (wx * e.ux + wy * e.uy) / (e.ux * e.ux + e.uy * e.uy);
    t = tmin(tmax(t, T(0.0)), T(1.0));
    T ex = wx - t * e.ux, ey = wy - t * e.uy;
    T d = sqrt(ex * ex + ey * ey);
    return on ? -d : d;
}

// Weights of the per-step metrics in a differentiable objective: element
// [k * N_tot + g] weighs agent g's metric at time t0+k+1; NULL = all 0.
struct MetricWeights { const double *logdiv, *ov, *off; };

template <class T> struct Objective { T loss, metrics; };

// The differentiable objective of one scene over nsteps steps, generic in
// the scalar type: the loss (squared log divergence plus the softplus
// overlap penalty) and, separately, the weighted sum of the per-step metrics
// of oracle_metrics (log divergence; overlap depth, the largest SAT depth
// against another valid agent; off-road distance, the largest signed
// distance over the box corners).  A metric of weight 0 is not evaluated; a
// metric of -inf (no other agent, no road edge) adds nothing.  IDM agents
// move as in oracle_transition but are constants for differentiation (their
// updates use the values only): the derivative flows through the policy
// agents' dynamics and every term.  st(g, c) gives component c (x, y,
// theta, vx, vy) of agent g's initial state.
template <class T, class ActFn, class StFn>
Objective<T> scene_objective(const ob_params* p, const ob_batch* b, int s, const ob_state* st0, StFn st,
                             ActFn act, int t0, int nsteps, double lambda, double tau, const MetricWeights* w) {
    const int a0 = b->agent_off[s], a1 = b->agent_off[s + 1], n = a1 - a0, N = b->N_tot;
    std::vector<St<T>> cur(n);
    std::vector<double> vals(6 * (size_t)n + 6);
    ob_state vs = {vals.data(), vals.data() + n, vals.data() + 2 * n, vals.data() + 3 * n,
                   vals.data() + 4 * n, vals.data() + 5 * n};
    for (int g = a0; g < a1; ++g) {
        cur[g - a0] = {st(g, 0), st(g, 1), st(g, 2), st(g, 3), st(g, 4)};
        vs.s[g - a0] = st0->s[g];
    }
    const bool with_metrics = w && (w->logdiv || w->ov || w->off);
    const std::vector<Seg> segs = with_metrics && w->off ? scene_segments(b, s) : std::vector<Seg>();
    T loss = T(0.0), metrics = T(0.0);
    std::vector<Box<T>> box(n);
    for (int k = 0; k < nsteps; ++k) {
        for (int g = a0; g < a1; ++g) {  // values of state t for the IDM agents
            vs.x[g - a0] = val(cur[g - a0].x); vs.y[g - a0] = val(cur[g - a0].y);
            vs.th[g - a0] = val(cur[g - a0].th); vs.vx[g - a0] = val(cur[g - a0].vx);
            vs.vy[g - a0] = val(cur[g - a0].vy);
        }
        std::vector<IdmOut> idm;
        for (int g = a0; g < a1; ++g)
            if (b->valid[g] && b->kind[g] == 2) idm.push_back(idm_agent(p, b, a0, a1, g, &vs, a0));
        size_t q = 0;
        for (int g = a0; g < a1; ++g) {
            if (!b->valid[g]) continue;
            if (b->kind[g] == 0) {
                cur[g - a0] = bicycle_forward(cur[g - a0], act(k, 0, g), act(k, 1, g), p->dt);
            } else if (b->kind[g] == 1) {
                cur[g - a0] = delta_forward(cur[g - a0], act(k, 0, g), act(k, 1, g), act(k, 2, g), p->dt);
            } else {
                const IdmOut& o = idm[q++];
                cur[g - a0] = {T(o.st.x), T(o.st.y), T(o.st.th), T(o.st.vx), T(o.st.vy)};
                vs.s[g - a0] = o.s;
            }
        }
        const int tl = t0 + k + 1;
        for (int g = a0; g < a1; ++g) {
            if (!b->valid[g]) continue;
            T dx = cur[g - a0].x - b->log_x[(size_t)tl * N + g];
            T dy = cur[g - a0].y - b->log_y[(size_t)tl * N + g];
            loss += dx * dx + dy * dy;
            box[g - a0] = make_box(cur[g - a0].x, cur[g - a0].y, cur[g - a0].th, b->L[g], b->W[g]);
        }
        for (int i = a0; i < a1; ++i) {
            if (!b->valid[i]) continue;
            for (int j = i + 1; j < a1; ++j) {
                if (!b->valid[j]) continue;
                T d = sat_depth(box[i - a0], box[j - a0]);
                loss += lambda * tau * softplus(d / tau);
            }
        }
        if (!with_metrics) continue;
        for (int g = a0; g < a1; ++g) {
            if (!b->valid[g]) continue;
            const size_t wi = (size_t)k * N + g;
            if (w->logdiv && w->logdiv[wi] != 0) {
                T dx = cur[g - a0].x - b->log_x[(size_t)tl * N + g];
                T dy = cur[g - a0].y - b->log_y[(size_t)tl * N + g];
                metrics += w->logdiv[wi] * sqrt(dx * dx + dy * dy);
            }
            if (w->ov && w->ov[wi] != 0) {
                T o = T(-kInf);
                for (int j = a0; j < a1; ++j) {
                    if (j == g || !b->valid[j]) continue;
                    const int lo = std::min(g, j), hi = std::max(g, j);
                    o = tmax(o, sat_depth(box[lo - a0], box[hi - a0]));
                }
                if (val(o) > -kInf) metrics += w->ov[wi] * o;
            }
            if (w->off && w->off[wi] != 0) {
                const Box<T>& B = box[g - a0];
                const double sl[4] = {1, 1, -1, -1}, sw[4] = {1, -1, -1, 1};
                T f = T(-kInf);
                for (int c = 0; c < 4; ++c) {
                    T px = B.cx + sl[c] * B.hl * B.c - sw[c] * B.hw * B.s;
                    T py = B.cy + sl[c] * B.hl * B.s + sw[c] * B.hw * B.c;
                    f = tmax(f, point_sd_t(segs, px, py));
                }
                if (val(f) > -kInf) metrics += w->off[wi] * f;
            }
        }
    }
    return {loss, metrics};
}

// The BPTT loss alone (no metric terms), from the initial state's values.
template <class T, class ActFn>
T scene_loss(const ob_params* p, const ob_batch* b, int s, const ob_state* st0, ActFn act,
             int t0, int nsteps, double lambda, double tau) {
    auto st = [&](int g, int c) {
        const double* f[5] = {st0->x, st0->y, st0->th, st0->vx, st0->vy};
        return T(f[c][g]);
    };
    return scene_objective<T>(p, b, s, st0, st, act, t0, nsteps, lambda, tau, nullptr).loss;
}

bool scene_differentiable(const ob_batch* b, int s) {
    for (int g = b->agent_off[s]; g < b->agent_off[s + 1]; ++g)
        if (b->valid[g] && b->kind[g] == 2 && b->route_off[g + 1] - b->route_off[g] < 2) return false;
    return true;
}

}  // namespace

extern "C" {

int oracle_transition(const ob_params* p, const ob_batch* b, int s0, int s1,
                      const ob_state* in, const double* act, const uint8_t* ctrl, int t_next,
                      ob_state* out, uint8_t* band_idm, int32_t* lead) {
    if (!p || !b || !in || !out || s0 < 0 || s1 > b->S || s0 > s1) return -1;
    for (int s = s0; s < s1; ++s)
        if (transition_scene(p, b, s, in, act, ctrl, t_next, out, band_idm, lead)) return -1;
    return 0;
}

int oracle_metrics(const ob_params* p, const ob_batch* b, int s0, int s1,
                   const ob_state* st, const ob_state* prev, int t, ob_metrics* m) {
    if (!p || !b || !st || !m || s0 < 0 || s1 > b->S || s0 > s1 || t < 0 || t >= b->T_log) return -1;
    for (int s = s0; s < s1; ++s)
        metrics_scene(p, b, s, st, prev, t, m->ov, m->off, m->logdiv, m->flags, m->reward);
    return 0;
}

int oracle_discretize(const ob_params* p, const ob_batch* b, const double* act, int T, int32_t* idx,
                      uint8_t* band) {
    if (!p || !b || !act || !idx || T < 0) return -1;
    const int N = b->N_tot;
    for (int k = 0; k < T; ++k)
        for (int g = 0; g < N; ++g) {
            const size_t o = (size_t)k * N + g;
            bool near = false;
            const double u[3] = {act[(k * 3 + 0) * (size_t)N + g], act[(k * 3 + 1) * (size_t)N + g],
                                 act[(k * 3 + 2) * (size_t)N + g]};
            idx[o] = b->valid[g] ? disc_encode(p, b->kind[g], u, &near) : -1;
            if (band) band[o] = near;
        }
    return 0;
}

int oracle_decode_actions(const ob_params* p, const ob_batch* b, const int32_t* idx, int T, double* act) {
    if (!p || !b || !act || !idx || T < 0) return -1;
    const int N = b->N_tot;
    for (int k = 0; k < T; ++k)
        for (int g = 0; g < N; ++g) {
            double u[3];
            disc_decode(p, b->kind[g], idx[(size_t)k * N + g], u);
            for (int c = 0; c < 3; ++c) act[(k * 3 + c) * (size_t)N + g] = u[c];
        }
    return 0;
}

int oracle_inverse(const ob_params* p, const ob_batch* b, int s0, int s1,
                   const ob_state* prev, const ob_state* next, double* act) {
    if (!p || !b || !prev || !next || !act || s0 < 0 || s1 > b->S || s0 > s1) return -1;
    const int N = b->N_tot;
    for (int g = b->agent_off[s0]; g < b->agent_off[s1]; ++g) {
        double u[3] = {0.0, 0.0, 0.0};
        if (b->valid[g]) inverse_action(p, b->kind[g], get_state(prev, g), get_state(next, g), u);
        for (int c = 0; c < 3; ++c) act[(size_t)c * N + g] = u[c];
    }
    return 0;
}

int oracle_expert_actions(const ob_params* p, const ob_batch* b, int s0, int s1, int t0, int T,
                          double* act_seq) {
    if (!p || !b || !act_seq || !has_full_log(b) || s0 < 0 || s1 > b->S || s0 > s1) return -1;
    if (t0 < 0 || T < 0 || t0 + T > b->T_log - 1) return -1;
    const int N = b->N_tot;
    for (int k = 0; k < T; ++k)
        for (int g = b->agent_off[s0]; g < b->agent_off[s1]; ++g) {
            double u[3] = {0.0, 0.0, 0.0};
            if (b->valid[g]) inverse_action(p, b->kind[g], log_state(b, t0 + k, g), log_state(b, t0 + k + 1, g), u);
            for (int c = 0; c < 3; ++c) act_seq[((size_t)k * 3 + c) * N + g] = u[c];
        }
    return 0;
}

int oracle_rollout(const ob_params* p, const ob_batch* b, int s0, int s1, ob_state* st,
                   const double* act_seq, const uint8_t* ctrl, int t0, int T, ob_metrics* mseq,
                   int nthreads) {
    if (!p || !b || !st || !mseq || s0 < 0 || s1 > b->S || s0 > s1) return -1;
    if (!act_seq && !ctrl) return -1;
    if (t0 < 0 || t0 + T > b->T_log - 1) return -1;
    const int N = b->N_tot, S = b->S;
    int status = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int s = s0; s < s1; ++s) {
        const int a0 = b->agent_off[s], a1 = b->agent_off[s + 1];
        // Scratch next-state arrays indexed by the global agent index.
        std::vector<double> buf(6 * (size_t)N);
        ob_state nxt = {buf.data(), buf.data() + N, buf.data() + 2 * N, buf.data() + 3 * N,
                        buf.data() + 4 * N, buf.data() + 5 * N};
        for (int k = 0; k < T; ++k) {
            const double* act = act_seq ? act_seq + (size_t)k * 3 * N : nullptr;
            if (transition_scene(p, b, s, st, act, ctrl, t0 + k + 1, &nxt, nullptr, nullptr)) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                status = -1;
                break;
            }
            size_t o = (size_t)k * N;
            metrics_scene(p, b, s, &nxt, st, t0 + k + 1, mseq->ov + o, mseq->off + o, mseq->logdiv + o,
                          mseq->flags + o, mseq->reward + (size_t)k * S);
            for (int g = a0; g < a1; ++g) copy_agent(&nxt, st, g);
        }
    }
    return status;
}

namespace {
// Nearest point of path q (points [k0, k1)) to (px, py): distance, arc length
// from the path's start, segment (ties: lower), and whether a non-adjacent
// segment lies within `band` of the nearest distance.
struct PathHit { double dist, arc; int seg; bool amb; };

PathHit path_nearest(const ob_batch* b, int k0, int k1, double px, double py, double band) {
    PathHit h{kInf, 0.0, -1, false};
    std::vector<double> d(std::max(k1 - k0 - 1, 0));
    double arc = 0.0;
    for (int k = k0; k + 1 < k1; ++k) {
        const double ax = b->path_x[k], ay = b->path_y[k];
        const double ux = b->path_x[k + 1] - ax, uy = b->path_y[k + 1] - ay;
        const double uu = ux * ux + uy * uy;
        const double t = uu > 0 ? std::min(1.0, std::max(0.0, ((px - ax) * ux + (py - ay) * uy) / uu)) : 0.0;
        const double ex = px - ax - t * ux, ey = py - ay - t * uy;
        const double dist = std::sqrt(ex * ex + ey * ey);
        d[k - k0] = dist;
        if (dist < h.dist) {
            h.dist = dist;
            h.arc = arc + t * std::sqrt(uu);
            h.seg = k - k0;
        }
        arc += std::sqrt(uu);
    }
    for (int j = 0; j < (int)d.size(); ++j)
        if (std::abs(j - h.seg) > 1 && d[j] - h.dist < band) h.amb = true;
    return h;
}
}  // namespace

int oracle_route(const ob_params* p, const ob_batch* b, int s0, int s1, const ob_state* st, double* progress,
                 uint8_t* flags) {
    if (!p || !b || !st || !progress || !flags || !b->path_off || s0 < 0 || s1 > b->S || s0 > s1) return -1;
    const int N = b->N_tot, TL = b->T_log;
    for (int s = s0; s < s1; ++s) {
        progress[s] = std::nan("");
        flags[s] = 0;
        const int g = b->agent_off[s];
        if (g >= b->agent_off[s + 1]) continue;
        int best = -1;
        PathHit on{kInf, 0, -1, false};
        double off = kInf, second_on = kInf;
        for (int q = b->path_off[s]; q < b->path_off[s + 1]; ++q) {
            const PathHit h = path_nearest(b, b->path_pt_off[q], b->path_pt_off[q + 1], st->x[g], st->y[g], p->band);
            if (b->path_on[q]) {
                if (h.dist < on.dist) {
                    second_on = on.dist;
                    on = h;
                    best = q;
                } else {
                    second_on = std::min(second_on, h.dist);
                }
            } else {
                off = std::min(off, h.dist);
            }
        }
        if (best < 0) continue;
        uint8_t fl = 0;
        if (on.dist > p->route_max_dist || on.dist - off > p->route_max_rel) fl |= 1;
        if (std::fabs(on.dist - p->route_max_dist) < p->band || std::fabs(on.dist - off - p->route_max_rel) < p->band)
            fl |= 2;
        if (on.amb || second_on - on.dist < p->band) fl |= 4;
        const int k0 = b->path_pt_off[best], k1 = b->path_pt_off[best + 1];
        const PathHit hp = path_nearest(b, k0, k1, b->log_x[g], b->log_y[g], p->band);
        const PathHit hq = path_nearest(b, k0, k1, b->log_x[(size_t)(TL - 1) * N + g], b->log_y[(size_t)(TL - 1) * N + g],
                                        p->band);
        if (hp.amb || hq.amb) fl |= 4;
        if (hq.arc - hp.arc > 1e-3) progress[s] = (on.arc - hp.arc) / (hq.arc - hp.arc);
        flags[s] = fl;
    }
    return 0;
}

int oracle_observe(const ob_params* p, const ob_batch* b, int s0, int s1, const ob_state* st,
                   const uint8_t* observers, int M, int K, double* agents, uint8_t* agents_valid,
                   double* rg, int32_t* rg_idx) {
    (void)p;
    if (!b || !st || !agents || !agents_valid || !rg || !rg_idx || K < 1 || s0 < 0 || s1 > b->S || s0 > s1)
        return -1;
    for (int s = s0; s < s1; ++s) {
        const int a0 = b->agent_off[s], a1 = b->agent_off[s + 1];
        const int r0 = b->rg_off[s], r1 = b->rg_off[s + 1];
        if (a1 - a0 > M) return -1;
        for (int g = a0; g < a1; ++g) {
            if (observers ? !observers[g] : !b->valid[g]) continue;
            const double cx = st->x[g], cy = st->y[g], th = st->th[g];
            const double c = std::cos(th), sn = std::sin(th);
            // Other agents in g's frame: rotate (p - c) by -theta_g.
            for (int j = 0; j < M; ++j) {
                double* o = agents + ((size_t)g * M + j) * 5;
                const int q = a0 + j;
                const bool ok = q < a1 && q != g && b->valid[q];
                agents_valid[(size_t)g * M + j] = ok;
                for (int k = 0; k < 5; ++k) o[k] = 0.0;
                if (!ok) continue;
                const double dx = st->x[q] - cx, dy = st->y[q] - cy;
                o[0] = c * dx + sn * dy;
                o[1] = -sn * dx + c * dy;
                o[2] = std::remainder(st->th[q] - th, kTwoPi);
                o[3] = c * st->vx[q] + sn * st->vy[q];
                o[4] = -sn * st->vx[q] + c * st->vy[q];
            }
            // The K nearest valid roadgraph points by the float32 key.
            const float fx = (float)cx, fy = (float)cy;
            std::vector<std::pair<float, int>> cand;
            for (int r = r0; r < r1; ++r) {
                if (!b->rg_valid[r]) continue;
                const float dxf = (float)b->rg_x[r] - fx, dyf = (float)b->rg_y[r] - fy;
                const float dyy = dyf * dyf;
                cand.push_back({std::fmaf(dxf, dxf, dyy), r});
            }
            std::sort(cand.begin(), cand.end());  // key, then index
            for (int k = 0; k < K; ++k) {
                double* o = rg + ((size_t)g * K + k) * 2;
                if (k < (int)cand.size()) {
                    const int r = cand[k].second;
                    const double dx = b->rg_x[r] - cx, dy = b->rg_y[r] - cy;
                    o[0] = c * dx + sn * dy;
                    o[1] = -sn * dx + c * dy;
                    rg_idx[(size_t)g * K + k] = r;
                } else {
                    o[0] = o[1] = 0.0;
                    rg_idx[(size_t)g * K + k] = -1;
                }
            }
        }
    }
    return 0;
}

double oracle_box_depth(const double* A, const double* B) {
    Box<double> a = make_box(A[0], A[1], A[2], A[3], A[4]);
    Box<double> c = make_box(B[0], B[1], B[2], B[3], B[4]);
    return sat_depth(a, c);
}

double oracle_point_sd(const ob_params* p, const ob_batch* b, int s, double px, double py,
                       int* ambiguous, int32_t* seg_out) {
    std::vector<Seg> g = scene_segments(b, s);
    int idx = -1;
    double r = point_sd(g, px, py, p->band, ambiguous, &idx);
    if (seg_out) *seg_out = idx >= 0 ? g[idx].k : -1;
    return r;
}

double oracle_loss(const ob_params* p, const ob_batch* b, int s, const ob_state* st0,
                   const double* act_seq, int t0, int T, double lambda, double tau) {
    if (!scene_differentiable(b, s) || t0 < 0 || t0 + T > b->T_log - 1) return std::nan("");
    const int N = b->N_tot;
    auto act = [&](int k, int c, int g) { return act_seq[((size_t)k * 3 + c) * N + g]; };
    return scene_loss<double>(p, b, s, st0, act, t0, T, lambda, tau);
}

int oracle_loss_grad(const ob_params* p, const ob_batch* b, int s, const ob_state* st0,
                     const double* act_seq, int t0, int T, double lambda, double tau, int n,
                     const int32_t* dir_t, const int32_t* dir_c, const int32_t* dir_g, double* grad) {
    if (!scene_differentiable(b, s) || t0 < 0 || t0 + T > b->T_log - 1) return -1;
    const int N = b->N_tot;
    for (int q = 0; q < n; ++q) {
        const int tq = dir_t[q], cq = dir_c[q], gq = dir_g[q];
        auto act = [&](int k, int c, int g) {
            double v = act_seq[((size_t)k * 3 + c) * N + g];
            return Dual(v, (k == tq && c == cq && g == gq) ? 1.0 : 0.0);
        };
        grad[q] = scene_loss<Dual>(p, b, s, st0, act, t0, T, lambda, tau).d;
    }
    return 0;
}

double oracle_objective(const ob_params* p, const ob_batch* b, int s, const ob_state* st0,
                        const double* act_seq, int t0, int T, double lambda, double tau, double w_loss,
                        const double* g_logdiv, const double* g_ov, const double* g_off) {
    if (!scene_differentiable(b, s) || t0 < 0 || t0 + T > b->T_log - 1) return std::nan("");
    const int N = b->N_tot;
    auto act = [&](int k, int c, int g) { return act_seq[((size_t)k * 3 + c) * N + g]; };
    auto st = [&](int g, int c) {
        const double* f[5] = {st0->x, st0->y, st0->th, st0->vx, st0->vy};
        return f[c][g];
    };
    const MetricWeights w = {g_logdiv, g_ov, g_off};
    const Objective<double> o = scene_objective<double>(p, b, s, st0, st, act, t0, T, lambda, tau, &w);
    return w_loss * o.loss + o.metrics;
}

int oracle_objective_grad(const ob_params* p, const ob_batch* b, int s, const ob_state* st0,
                          const double* act_seq, int t0, int T, double lambda, double tau, double w_loss,
                          const double* g_logdiv, const double* g_ov, const double* g_off, int n,
                          const int32_t* dir_kind, const int32_t* dir_t, const int32_t* dir_c,
                          const int32_t* dir_g, double* grad) {
    if (!scene_differentiable(b, s) || t0 < 0 || t0 + T > b->T_log - 1) return -1;
    const int N = b->N_tot;
    const MetricWeights w = {g_logdiv, g_ov, g_off};
    for (int q = 0; q < n; ++q) {
        const int kq = dir_kind[q], tq = dir_t[q], cq = dir_c[q], gq = dir_g[q];
        if (kq < 0 || kq > 1 || cq < 0 || cq > (kq == 0 ? 2 : 4) || gq < 0 || gq >= N) return -1;
        auto act = [&](int k, int c, int g) {
            const double v = act_seq[((size_t)k * 3 + c) * N + g];
            return Dual(v, (kq == 0 && k == tq && c == cq && g == gq) ? 1.0 : 0.0);
        };
        auto st = [&](int g, int c) {
            const double* f[5] = {st0->x, st0->y, st0->th, st0->vx, st0->vy};
            return Dual(f[c][g], (kq == 1 && g == gq && c == cq) ? 1.0 : 0.0);
        };
        const Objective<Dual> o = scene_objective<Dual>(p, b, s, st0, st, act, t0, T, lambda, tau, &w);
        grad[q] = w_loss * o.loss.d + o.metrics.d;
    }
    return 0;
}

}  // extern "C"
