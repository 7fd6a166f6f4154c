/*
 * npp_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * per-sampling-time batched rollout of Plessen, "Online Sampling in the
 * Parameter Space of a Neural Network for GPU-accelerated Motion Planning
 * of Autonomous Vehicles" (arXiv 1904.06680).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) never calls it, and the two share no code: this file
 * includes no project header and is compiled on its own.
 *
 * Precision: FP64 everywhere except the parameter sampler (Philox4x32-10
 * followed by the FP32 Box-Muller specification "Normal32"), whose FP32
 * operation sequence is part of the method's definition here and is emulated
 * bit-for-bit; the sampled FP32 values are then promoted to double.
 * Compile with -ffp-contract=off so that no multiply-add is fused behind the
 * code's back (fmaf() is used explicitly where the specification fuses).
 *
 * What each function follows (paper sections / equations):
 *   philox4x32_10     Salmon et al., SC'11 (the counter-based generator; the
 *                     paper only says a random seed is passed per sampling
 *                     time, Sect. II-D "Fourth")
 *   orc_normal_pair   Box-Muller on two 23-bit uniforms, FP32 spec Normal32
 *   orc_frame_to_ev   obstacle data in the EV-aligned (xi, eta) frame,
 *                     Sect. II-C (measurements m^ext)
 *   features()        feature vector s_{t+h}, Eq. (eq_def_stph), plus three
 *                     project features for the 8-input networks
 *   mlp()             multilayer perceptron a = X(s, theta), Eq. (eq_def_at),
 *                     tanh on every layer
 *   euler_step()      kinematic bicycle model, Sect. IV "Vehicle model",
 *                     explicit Euler on the old state with step Ts
 *   collides()        polytope check A(phi)(p_j(h) - [x,y]) < b(phi), Eq.
 *                     (eq_Apsietc_collAvoidIneqs), obstacle points extrapolated
 *                     at constant velocity, Sect. II-D items (i)-(iv)
 *   orc_plan          best of N sampled rollouts (one TSHC sampling batch,
 *                     Sect. II-D "Fifth"/"Sixth"), lowest index on ties;
 *                     optionally the first n_prop samples drawn from a
 *                     Gaussian proposal (mean, std) instead of N(0, I)
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors; Normal32
 * against FP64 libm Box-Muller and moment/KS checks; the Fig. 3 state table
 * of the paper replayed step by step; straight-line and circular-arc closed
 * forms of the Euler recurrence; brute-force point-in-rectangle by corner
 * cross products; rigid-motion invariance; brute-force argmin; MLP layout
 * against numpy matmul on the declared parameter order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* configuration (FP64)                                                 */
/* ------------------------------------------------------------------ */
#define ORC_MAX_LAYERS 8

typedef struct {
    /* kinematic bicycle, Sect. IV "Vehicle model", Table veh */
    double lf, lr;            /* CoG to front / rear axle [m]            */
    double delta_max;         /* max steering angle [rad]                */
    double delta_rate_max;    /* max steering rate [rad/s]               */
    double u_min, u_max;      /* longitudinal acceleration range [m/s^2] */
    double Ts;                /* sampling time [s]                       */
    /* rectangular footprint relative to the reference point */
    double half_len, half_wid, c_off;
    /* feature normalisation, Table hyperparameters */
    double dxi_n, deta_n, dphi_n, dv_n;
    /* cost weights (reading: the paper gives no cost) */
    double w_pos, w_phi, w_v, w_effort;
    /* network: widths[0] = inputs, widths[n_layers] = 2 outputs */
    int32_t n_layers;
    int32_t widths[ORC_MAX_LAYERS + 1];
    /* variants (Sect. V): goal offsets of the features in the body frame at
     * t+h instead of the EV frame at t; velocity constraints imposed by
     * discarding every sample whose speed leaves [v_min, v_max] */
    int32_t feature_frame;    /* 0: EV frame at t, 1: body frame at t+h */
    int32_t v_limits;         /* 1: speed limits on                     */
    double v_min, v_max;      /* [m/s]                                  */
    /* general footprint (Sect. II-D: the EV as an arbitrarily refined
     * polytope, convex or not): the union of fp_pieces convex polygons, each
     * given by its vertices counter-clockwise in the vehicle's frame (x along
     * the heading, origin at the reference point).  0 pieces: the rectangle
     * above. */
    int32_t fp_pieces;
    const int32_t* fp_start;  /* [fp_pieces + 1] first vertex of each piece */
    const double* fp_verts;   /* [fp_start[fp_pieces]][2]                */
} orc_config;

enum { ORC_OK = 0, ORC_INFEASIBLE = 2, ORC_INVALID = 1 };

int orc_n_theta(const orc_config* c)
{
    int n = 0;
    for (int l = 0; l < c->n_layers; ++l)
        n += c->widths[l + 1] * c->widths[l] + c->widths[l + 1];
    return n;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                    */
/* ------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* multipliers   */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key bumps */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Normal32: the FP32 Box-Muller specification                          */
/* ------------------------------------------------------------------ */
static float f_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* u = (2*(w >> 9) + 1) * 2^-24: an odd multiple of 2^-24 in (0, 1), exact */
float orc_u24(uint32_t w)
{
    uint32_t K = ((w >> 9) << 1) | 1u;
    return (float)K * 0x1p-24f;
}

/* natural log for u in (0,1): u = 2^e f, f in [sqrt(1/2), sqrt(2)),
 * ln f = 2 atanh(s), s = (f-1)/(f+1), odd Taylor series to s^11. */
float orc_ln32(float u)
{
    uint32_t b = bits_from_f(u);
    int e = (int)(b >> 23) - 127;
    uint32_t m = b & 0x7FFFFFu;
    float f;
    if (m > 0x3504F3u) { f = f_from_bits(m | 0x3F000000u); e += 1; }
    else               { f = f_from_bits(m | 0x3F800000u); }
    float num = f - 1.0f;               /* exact (Sterbenz)          */
    float den = f + 1.0f;
    float s = num / den;
    float z = s * s;
    float p = fmaf(z, 0x1.745d18p-3f, 0x1.c71c72p-3f);   /* 2/11, 2/9 */
    p = fmaf(z, p, 0x1.24924ap-2f);                       /* 2/7       */
    p = fmaf(z, p, 0x1.99999ap-2f);                       /* 2/5       */
    p = fmaf(z, p, 0x1.555556p-1f);                       /* 2/3       */
    float t = s * z;
    float lnf = fmaf(t, p, 2.0f * s);
    float ef = (float)e;
    const float LN2_HI = 0x1.62e400p-1f;   /* ln 2 with 9 trailing zero bits */
    const float LN2_LO = 0x1.7f7d1cp-20f;  /* RN(ln 2 - LN2_HI)              */
    return fmaf(ef, LN2_HI, fmaf(ef, LN2_LO, lnf));
}

/* sin and cos of 2*pi*u for u = K * 2^-24, K odd in [1, 2^24):
 * quarter-turn reduction in integers, Taylor polynomials on |x| <= pi/4. */
void orc_sincos2pi32(uint32_t K, float* s_out, float* c_out)
{
    int32_t q = (int32_t)((K + (1u << 21)) >> 22);       /* round(4u)   */
    int32_t k = (int32_t)K - q * (1 << 22);               /* |k| <= 2^21 */
    float x = (float)k * 0x1.921fb6p-22f;                 /* RN(2pi) 2^-24 */
    float z = x * x;
    float ps = fmaf(z, 0x1.71de3ap-19f, -0x1.a01a02p-13f); /* 1/9!, -1/7! */
    ps = fmaf(z, ps, 0x1.111112p-7f);                      /* 1/5!        */
    ps = fmaf(z, ps, -0x1.555556p-3f);                     /* -1/3!       */
    float sx = fmaf(x * z, ps, x);
    float pc = fmaf(z, -0x1.27e4fcp-22f, 0x1.a01a02p-16f); /* -1/10!, 1/8! */
    pc = fmaf(z, pc, -0x1.6c16c2p-10f);                    /* -1/6!       */
    pc = fmaf(z, pc, 0x1.555556p-5f);                      /* 1/4!        */
    pc = fmaf(z, pc, -0.5f);                               /* -1/2!       */
    float cx = fmaf(z, pc, 1.0f);
    switch (q & 3) {
    case 0: *s_out = sx;  *c_out = cx;  break;
    case 1: *s_out = cx;  *c_out = -sx; break;
    case 2: *s_out = -sx; *c_out = -cx; break;
    default: *s_out = -cx; *c_out = sx; break;
    }
}

/* Box-Muller: radius from word a, angle from word b -> (R cos, R sin) */
void orc_normal_pair(uint32_t a, uint32_t b, float out[2])
{
    float u1 = orc_u24(a);
    float r = sqrtf(-2.0f * orc_ln32(u1));
    uint32_t K = ((b >> 9) << 1) | 1u;
    float s, c;
    orc_sincos2pi32(K, &s, &c);
    out[0] = r * c;
    out[1] = r * s;
}

/* theta_n[i] from Philox(ctr = (i/4, n, t_index, stream), key = seed):
 * words (0,1) give theta[4q], theta[4q+1]; words (2,3) give 4q+2, 4q+3. */
void orc_theta(uint64_t seed, uint32_t t_index, uint32_t stream, uint32_t n,
               int n_theta, float* out)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int q = 0; 4 * q < n_theta; ++q) {
        uint32_t ctr[4] = { (uint32_t)q, n, t_index, stream }, w[4];
        orc_philox(ctr, key, w);
        float z[4];
        orc_normal_pair(w[0], w[1], z);
        orc_normal_pair(w[2], w[3], z + 2);
        for (int j = 0; j < 4 && 4 * q + j < n_theta; ++j) out[4 * q + j] = z[j];
    }
}

/* ------------------------------------------------------------------ */
/* geometry: world frame <-> EV-aligned frame at time t                 */
/* ------------------------------------------------------------------ */
/* state_w = (x, y, phi, v, a_prev0, a_prev1); goal_w = (x, y, phi, v);
 * obs_w[M][4] = (x, y, vx, vy).  Output goal_ev[4], obs_ev[M][4]. */
void orc_frame_to_ev(const double* state_w, const double* goal_w,
                     const double* obs_w, int M, double* goal_ev, double* obs_ev)
{
    double c = cos(state_w[2]), s = sin(state_w[2]);
    double dx = goal_w[0] - state_w[0], dy = goal_w[1] - state_w[1];
    goal_ev[0] = c * dx + s * dy;
    goal_ev[1] = -s * dx + c * dy;
    goal_ev[2] = goal_w[2] - state_w[2];
    goal_ev[3] = goal_w[3];
    for (int j = 0; j < M; ++j) {
        const double* p = obs_w + 4 * j;
        double* q = obs_ev + 4 * j;
        double px = p[0] - state_w[0], py = p[1] - state_w[1];
        q[0] = c * px + s * py;
        q[1] = -s * px + c * py;
        q[2] = c * p[2] + s * p[3];
        q[3] = -s * p[2] + c * p[3];
    }
}

static void ev_to_world(const double* state_w, const double z_ev[4], double* z_w)
{
    double c = cos(state_w[2]), s = sin(state_w[2]);
    z_w[0] = state_w[0] + c * z_ev[0] - s * z_ev[1];
    z_w[1] = state_w[1] + s * z_ev[0] + c * z_ev[1];
    z_w[2] = state_w[2] + z_ev[2];
    z_w[3] = z_ev[3];
}

/* wrap an angle into [-pi, pi) */
static double wrap_pi(double a)
{
    const double TWO_PI = 2.0 * M_PI;
    return a - TWO_PI * floor((a + M_PI) / TWO_PI);
}

/* ------------------------------------------------------------------ */
/* the rollout pieces                                                   */
/* ------------------------------------------------------------------ */

/* Eq. (eq_def_stph): deviations from the goal in the EV-aligned frame at t,
 * normalised by the Delta constants, and the last applied steering.  For
 * 8-input networks three more entries follow: last applied acceleration
 * command, normalised speed, and the remaining-horizon fraction.  With
 * feature_frame = 1 the position deviation is expressed in the vehicle's
 * own frame at t+h (rotated by -phi_{t+h}), the variant Sect. V names. */
void orc_features(const orc_config* c, const double z[4], const double ap[2],
                  const double goal[4], int h, int T, double* s)
{
    double dx = goal[0] - z[0], dy = goal[1] - z[1];
    if (c->feature_frame == 1) {
        double cp = cos(z[2]), sp = sin(z[2]);
        double bx = cp * dx + sp * dy, by = -sp * dx + cp * dy;
        dx = bx;
        dy = by;
    }
    s[0] = dx / c->dxi_n;
    s[1] = dy / c->deta_n;
    s[2] = wrap_pi(goal[2] - z[2]) / c->dphi_n;
    s[3] = (goal[3] - z[3]) / c->dv_n;
    s[4] = ap[0];
    if (c->widths[0] == 8) {
        s[5] = ap[1];
        s[6] = z[3] / c->dv_n;
        s[7] = (double)(T - h) / (double)T;
    }
}

/* standard multilayer perceptron, tanh on every layer; parameter order per
 * layer: W[out][in] row-major, then b[out]. */
void orc_mlp(const orc_config* c, const double* theta, const double* s, double* a)
{
    double buf0[256], buf1[256];
    const double* in = s;
    double* out = buf0;
    const double* p = theta;
    for (int l = 0; l < c->n_layers; ++l) {
        int ni = c->widths[l], no = c->widths[l + 1];
        const double* W = p;
        const double* b = p + no * ni;
        for (int o = 0; o < no; ++o) {
            double acc = b[o];
            for (int i = 0; i < ni; ++i) acc += W[o * ni + i] * in[i];
            out[o] = tanh(acc);
        }
        p += no * ni + no;
        in = out;
        out = (out == buf0) ? buf1 : buf0;
    }
    a[0] = in[0];
    a[1] = in[1];
}

/* network output -> applied normalised controls: the steering command moves
 * at most delta_rate_max*Ts/delta_max per step (Table veh; Figs. 3 and 8) and
 * stays in [-1, 1]; the acceleration command is used as is. */
void orc_controls(const orc_config* c, const double a_raw[2], const double ap[2],
                  double* a_applied)
{
    double r = c->delta_rate_max * c->Ts / c->delta_max;
    double a0 = a_raw[0];
    if (a0 < ap[0] - r) a0 = ap[0] - r;
    if (a0 > ap[0] + r) a0 = ap[0] + r;
    if (a0 < -1.0) a0 = -1.0;
    if (a0 > 1.0) a0 = 1.0;
    a_applied[0] = a0;
    a_applied[1] = a_raw[1];
}

/* kinematic bicycle (Sect. IV), delta = delta_max a0,
 * u = u_min + (a1+1)/2 (u_max - u_min), one explicit Euler step of length Ts
 * evaluated on the old state. */
void orc_euler_step(const orc_config* c, const double z[4], const double a[2], double* zn)
{
    double L = c->lf + c->lr;
    double delta = c->delta_max * a[0];
    double u = c->u_min + 0.5 * (a[1] + 1.0) * (c->u_max - c->u_min);
    double beta = atan(c->lr * tan(delta) / L);
    double x = z[0], y = z[1], phi = z[2], v = z[3];
    zn[0] = x + c->Ts * v * cos(phi + beta) / cos(beta);
    zn[1] = y + c->Ts * v * sin(phi + beta) / cos(beta);
    zn[2] = phi + c->Ts * v * tan(delta) / L;
    zn[3] = v + c->Ts * u;
}

/* Eq. (eq_Apsietc_collAvoidIneqs) for a rectangle: rows of A(phi) are the
 * outward face normals, b(phi) the face offsets from the reference point.
 * Obstacle j at time t+h is p_j + tau v_j (constant velocity, tau = h Ts).
 * Returns 1 when some point satisfies all four strict inequalities.  When
 * n_clear / n_near are given, also counts points that are inside by more
 * than `margin` and points whose decision lies within `margin` of a face. */
static int collide_footprint(const orc_config* c, double x, double y, double phi,
                             const double* obs_ev, int M, double tau, double margin,
                             int* n_clear, int* n_near);

int orc_collide(const orc_config* c, double x, double y, double phi,
                const double* obs_ev, int M, double tau, double margin,
                int* n_clear, int* n_near)
{
    if (c->fp_pieces > 0)
        return collide_footprint(c, x, y, phi, obs_ev, M, tau, margin, n_clear, n_near);
    double cp = cos(phi), sp = sin(phi);
    double A[4][2] = { { cp, sp }, { -cp, -sp }, { -sp, cp }, { sp, -cp } };
    double b[4] = { c->c_off + c->half_len, c->half_len - c->c_off,
                    c->half_wid, c->half_wid };
    int hit = 0, clear = 0, near = 0;
    for (int j = 0; j < M; ++j) {
        const double* p = obs_ev + 4 * j;
        double dx = p[0] + tau * p[2] - x;
        double dy = p[1] + tau * p[3] - y;
        double worst = -INFINITY;       /* max_i (A d - b)_i */
        int inside = 1;
        for (int i = 0; i < 4; ++i) {
            double g = A[i][0] * dx + A[i][1] * dy - b[i];
            if (!(g < 0.0)) inside = 0;
            if (g > worst) worst = g;
        }
        if (inside) hit = 1;
        if (worst < -margin) clear++;
        else if (worst <= margin) near++;
        if (hit && !n_clear && !n_near) return 1;
    }
    if (n_clear) *n_clear = clear;
    if (n_near) *n_near = near;
    return hit;
}

/* The same check for a general footprint: point j at time t+h is moved into
 * the vehicle's frame, q = R(-phi) (p_j(h) - [x, y]), and is inside a convex
 * piece when it lies strictly to the left of every directed edge v_i ->
 * v_{i+1} of that counter-clockwise polygon (cross product > 0); a
 * collision is a point inside some piece.  For the margin counts a point's
 * depth is the largest over pieces of its smallest distance to an edge line
 * (positive inside). */
static int collide_footprint(const orc_config* c, double x, double y, double phi,
                             const double* obs_ev, int M, double tau, double margin,
                             int* n_clear, int* n_near)
{
    double cp = cos(phi), sp = sin(phi);
    int hit = 0, clear = 0, near = 0;
    for (int j = 0; j < M; ++j) {
        const double* p = obs_ev + 4 * j;
        double dx = p[0] + tau * p[2] - x;
        double dy = p[1] + tau * p[3] - y;
        double qx = cp * dx + sp * dy, qy = -sp * dx + cp * dy;
        double depth = -INFINITY;
        int inside_any = 0;
        for (int k = 0; k < c->fp_pieces; ++k) {
            int b = c->fp_start[k], e = c->fp_start[k + 1], n = e - b;
            int inside = 1;
            double dmin = INFINITY;
            for (int i = 0; i < n; ++i) {
                const double* v0 = c->fp_verts + 2 * (b + i);
                const double* v1 = c->fp_verts + 2 * (b + (i + 1) % n);
                double ex = v1[0] - v0[0], ey = v1[1] - v0[1];
                double cr = ex * (qy - v0[1]) - ey * (qx - v0[0]);
                if (!(cr > 0.0)) inside = 0;
                double d = cr / hypot(ex, ey);
                if (d < dmin) dmin = d;
            }
            if (inside) inside_any = 1;
            if (dmin > depth) depth = dmin;
        }
        if (inside_any) hit = 1;
        if (depth > margin) clear++;
        else if (depth >= -margin) near++;
        if (hit && !n_clear && !n_near) return 1;
    }
    if (n_clear) *n_clear = clear;
    if (n_near) *n_near = near;
    return hit;
}

/* Velocity constraints by discarding samples (Sect. V): a state reached by
 * the sample's own controls (h >= 1) whose speed is outside [v_min, v_max]
 * ends the sample there as a collision does.  The initial speed is given,
 * not chosen, so h = 0 is never discarded for it. */
int orc_speed_violated(const orc_config* c, double v, int h)
{
    return c->v_limits == 1 && h > 0 && !(v >= c->v_min && v <= c->v_max);
}

/* ------------------------------------------------------------------ */
/* one rollout                                                          */
/* ------------------------------------------------------------------ */
/* Cost of a collision-free rollout (the reading of the cost: the paper
 * gives none): pose distance of the final EV-frame state z to the goal plus
 * the mean squared normalised control, E = sum over the T applied controls
 * of a0^2 + a1^2. */
static double terminal_cost(const orc_config* c, const double z[4], double E, int T, const double goal[4])
{
    double dpos = hypot(z[0] - goal[0], z[1] - goal[1]);
    return c->w_pos * dpos + c->w_phi * fabs(wrap_pi(z[2] - goal[2]))
         + c->w_v * fabs(z[3] - goal[3]) + c->w_effort * E / (double)T;
}

/* The cost of a collision-free rollout from its final state zT and its
 * applied controls ctrl[T][2] (for instance a GPU rollout's own FP32 rows,
 * so that the cost is checked at the GPU's states). */
double orc_cost(const orc_config* c, const double zT[4], const double* ctrl, int T, const double goal[4])
{
    double E = 0.0;
    for (int h = 0; h < T; ++h) E += ctrl[2 * h] * ctrl[2 * h] + ctrl[2 * h + 1] * ctrl[2 * h + 1];
    return terminal_cost(c, zT, E, T, goal);
}

/* z0 = EV-frame state (x, y, phi, v) (normally (0,0,0,v0)), ap0 = last
 * applied controls, goal/obs in the EV frame.  traj[(T+1)][4] and
 * ctrl[T][2] in the EV frame; for a collided sample rows after the first
 * collision repeat the collided state and the controls there are zero.
 * Returns first_hit (-1 when collision-free) and writes the cost. */
static int rollout(const orc_config* c, const double* theta, const double z0[4],
                   const double ap0[2], const double goal[4], const double* obs,
                   int M, int T, double* cost, double* traj, double* ctrl)
{
    double z[4] = { z0[0], z0[1], z0[2], z0[3] };
    double ap[2] = { ap0[0], ap0[1] };
    double E = 0.0;
    int fh = -1;
    for (int h = 0; h <= T; ++h) {
        if (traj) memcpy(traj + 4 * h, z, sizeof z);
        if (orc_speed_violated(c, z[3], h) ||
            orc_collide(c, z[0], z[1], z[2], obs, M, h * c->Ts, 0.0, NULL, NULL)) {
            fh = h;
            break;
        }
        if (h == T) break;
        double s[16], araw[2], a[2], zn[4];
        orc_features(c, z, ap, goal, h, T, s);
        orc_mlp(c, theta, s, araw);
        orc_controls(c, araw, ap, a);
        E += a[0] * a[0] + a[1] * a[1];
        if (ctrl) { ctrl[2 * h] = a[0]; ctrl[2 * h + 1] = a[1]; }
        orc_euler_step(c, z, a, zn);
        memcpy(z, zn, sizeof z);
        ap[0] = a[0];
        ap[1] = a[1];
    }
    if (fh >= 0) {
        if (traj) for (int h = fh + 1; h <= T; ++h) memcpy(traj + 4 * h, traj + 4 * fh, 4 * sizeof(double));
        if (ctrl) for (int h = fh; h < T; ++h) { ctrl[2 * h] = 0.0; ctrl[2 * h + 1] = 0.0; }
        *cost = INFINITY;
    } else {
        *cost = terminal_cost(c, z, E, T, goal);
    }
    return fh;
}

/* one replay step from a given (possibly FP32) state: the applied controls
 * and the next state, as the rollout computes them at horizon index h. */
void orc_step(const orc_config* c, const double* theta, const double z[4],
              const double ap[2], const double goal_ev[4], int h, int T,
              double* a_out, double* zn)
{
    double s[16], araw[2];
    orc_features(c, z, ap, goal_ev, h, T, s);
    orc_mlp(c, theta, s, araw);
    orc_controls(c, araw, ap, a_out);
    orc_euler_step(c, z, a_out, zn);
}

static void sample_theta(const orc_config* c, uint64_t seed, uint32_t t_index,
                         uint32_t stream, uint32_t n, double* theta, float* tmp)
{
    int nt = orc_n_theta(c);
    orc_theta(seed, t_index, stream, n, nt, tmp);
    for (int i = 0; i < nt; ++i) theta[i] = (double)tmp[i];
}

/* Sample n of a plan step with a sampling proposal (mean mu, standard
 * deviation sigma, both FP32): samples n < n_prop are mu + sigma * eps with
 * eps the normals of stream prop_stream (1 for the learned proposal, r for
 * restart round r of the hill climb), rounded once to FP32 (a fused multiply-add,
 * C99 fmaf, correctly rounded); the others are the isotropic samples of the
 * given stream.  With n_prop = 0 this is sample_theta. */
static void sample_theta_mixed(const orc_config* c, uint64_t seed, uint32_t t_index,
                               uint32_t stream, uint32_t n, const float* mu, const float* sigma,
                               int n_prop, uint32_t prop_stream, double* theta, float* tmp)
{
    if ((int64_t)n >= (int64_t)n_prop || !mu || !sigma) {
        sample_theta(c, seed, t_index, stream, n, theta, tmp);
        return;
    }
    int nt = orc_n_theta(c);
    orc_theta(seed, t_index, prop_stream, n, nt, tmp);
    for (int i = 0; i < nt; ++i) theta[i] = (double)fmaf(sigma[i], tmp[i], mu[i]);
}

/* Rollouts of explicit parameter vectors theta[K][n_theta] (EV-frame inputs).
 * Outputs per sample: cost[K], first_hit[K], and if non-NULL
 * traj[K][T+1][4], ctrl[K][T][2] (EV frame). */
void orc_rollout_theta(const orc_config* c, const double* theta, int K,
                       const double z0[4], const double ap0[2], const double* goal_ev,
                       const double* obs_ev, int M, int T, int n_threads,
                       double* cost, int32_t* first_hit, double* traj, double* ctrl)
{
    int nt = orc_n_theta(c);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int k = 0; k < K; ++k) {
        first_hit[k] = rollout(c, theta + (size_t)k * nt, z0, ap0, goal_ev, obs_ev, M, T,
                               cost + k, traj ? traj + (size_t)k * (T + 1) * 4 : NULL,
                               ctrl ? ctrl + (size_t)k * T * 2 : NULL);
    }
}

/* Rollouts of Philox-sampled samples idx[K] (EV-frame inputs); warm, when
 * non-NULL, replaces sample 0's parameters. */
/* theta_n of a plan step with a proposal (FP32 values, see
 * sample_theta_mixed) */
void orc_theta_mixed(uint64_t seed, uint32_t t_index, uint32_t n, int n_theta, const float* mu,
                     const float* sigma, int n_prop, uint32_t prop_stream, float* out)
{
    if ((int64_t)n >= (int64_t)n_prop || !mu || !sigma) {
        orc_theta(seed, t_index, 0u, n, n_theta, out);
        return;
    }
    orc_theta(seed, t_index, prop_stream, n, n_theta, out);
    for (int i = 0; i < n_theta; ++i) out[i] = fmaf(sigma[i], out[i], mu[i]);
}

void orc_rollout_samples(const orc_config* c, uint64_t seed, uint32_t t_index,
                         uint32_t stream, const int32_t* idx, int K, const double* warm,
                         const float* mu, const float* sigma, int n_prop, uint32_t prop_stream,
                         const double z0[4], const double ap0[2], const double* goal_ev,
                         const double* obs_ev, int M, int T, int n_threads,
                         double* cost, int32_t* first_hit, double* traj, double* ctrl)
{
    int nt = orc_n_theta(c);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double* theta = (double*)malloc(sizeof(double) * nt);
        float* tmp = (float*)malloc(sizeof(float) * (nt + 4));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int k = 0; k < K; ++k) {
            if (warm && idx[k] == 0) memcpy(theta, warm, sizeof(double) * nt);
            else sample_theta_mixed(c, seed, t_index, stream, (uint32_t)idx[k], mu, sigma, n_prop,
                                    prop_stream, theta, tmp);
            first_hit[k] = rollout(c, theta, z0, ap0, goal_ev, obs_ev, M, T, cost + k,
                                   traj ? traj + (size_t)k * (T + 1) * 4 : NULL,
                                   ctrl ? ctrl + (size_t)k * T * 2 : NULL);
        }
        free(theta);
        free(tmp);
    }
}

/* ------------------------------------------------------------------ */
/* plan: best of N sampled rollouts                                     */
/* ------------------------------------------------------------------ */
/* World-frame inputs.  Writes costs[N], first_hit[N] (if non-NULL), and the
 * winner: index, status (OK, or INFEASIBLE when every sample collided, in
 * which case the winner is the sample that survived longest, lowest index
 * on ties), cost, parameters [n_theta], controls [T][2] and trajectory
 * [T+1][4] in the world frame. */
int orc_plan(const orc_config* c, const double* state_w, const double* goal_w,
             const double* obs_w, int M, int N, int T, uint64_t seed,
             uint32_t t_index, const double* warm, const float* mu, const float* sigma,
             int n_prop, uint32_t prop_stream, int n_threads,
             double* costs, int32_t* first_hit, int32_t* best_idx, int32_t* status,
             double* best_cost, double* best_theta, double* controls, double* traj_w)
{
    if (N <= 0 || T <= 0 || M < 0) return ORC_INVALID;
    int nt = orc_n_theta(c);
    double goal_ev[4];
    double* obs_ev = (double*)malloc(sizeof(double) * 4 * (M > 0 ? M : 1));
    orc_frame_to_ev(state_w, goal_w, obs_w, M, goal_ev, obs_ev);
    double z0[4] = { 0.0, 0.0, 0.0, state_w[3] };
    double ap0[2] = { state_w[4], state_w[5] };
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * N);
    double* cst = (double*)malloc(sizeof(double) * N);
    int32_t* fh = (int32_t*)malloc(sizeof(int32_t) * N);
    for (int n = 0; n < N; ++n) idx[n] = n;
    orc_rollout_samples(c, seed, t_index, 0u, idx, N, warm, mu, sigma, n_prop, prop_stream, z0, ap0,
                        goal_ev, obs_ev, M, T, n_threads, cst, fh, NULL, NULL);
    /* argmin over collision-free samples, lowest index on ties */
    int best = -1;
    for (int n = 0; n < N; ++n)
        if (fh[n] < 0 && (best < 0 || cst[n] < cst[best])) best = n;
    int st = ORC_OK;
    if (best < 0) {          /* all collided: longest survivor */
        st = ORC_INFEASIBLE;
        best = 0;
        for (int n = 1; n < N; ++n) if (fh[n] > fh[best]) best = n;
    }
    if (costs) memcpy(costs, cst, sizeof(double) * N);
    if (first_hit) memcpy(first_hit, fh, sizeof(int32_t) * N);
    *best_idx = best;
    *status = st;
    *best_cost = cst[best];
    /* re-roll the winner for its controls and trajectory */
    double* theta = (double*)malloc(sizeof(double) * nt);
    float* tmp = (float*)malloc(sizeof(float) * (nt + 4));
    if (warm && best == 0) memcpy(theta, warm, sizeof(double) * nt);
    else sample_theta_mixed(c, seed, t_index, 0u, (uint32_t)best, mu, sigma, n_prop, prop_stream, theta, tmp);
    if (best_theta) memcpy(best_theta, theta, sizeof(double) * nt);
    double* traj_ev = (double*)malloc(sizeof(double) * 4 * (T + 1));
    double dummy;
    rollout(c, theta, z0, ap0, goal_ev, obs_ev, M, T, &dummy, traj_ev, controls);
    if (traj_w)
        for (int h = 0; h <= T; ++h) ev_to_world(state_w, traj_ev + 4 * h, traj_w + 4 * h);
    free(traj_ev); free(theta); free(tmp);
    free(idx); free(cst); free(fh); free(obs_ev);
    return st;
}
