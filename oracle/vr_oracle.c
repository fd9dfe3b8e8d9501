/*
 * vr_oracle.c -- plain, slow, FP64 CPU reference of the direct volume ray caster
 * described in N. Kopal, "Volume Raycasting mit OpenCL" (2011), arXiv:1609.01317.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant table with the CUDA implementation.
 *
 * What it computes (section / equation numbers are those of the paper):
 *   - Eq. 1 (§2.1): a volume is a function on the integer grid; voxel (x,y,z) sits at
 *     world point (x,y,z) with unit spacing.
 *   - §3.3 / §3.6: one ray per pixel, intersected with a bounding box (the clip box
 *     intersected with the volume box [0,n-1]^3); no hit -> black (RGBA 0); samples at
 *     regular spacing between entry and exit (midpoint rule, see below).
 *   - Eq. 2 + §3.4: trilinear interpolation as nested linear interpolations.
 *   - Eq. 3 (§3.5): central differences; Eq. 4 (§3.5): Sobel3D masks; §3.5 / §4: the
 *     Zucker-Hummel operator (54 taps, mask not printed in the paper).
 *   - §3.7: colour / opacity from a lookup table indexed by the voxel value.
 *   - §3.8 + Listing 3: point-light shading from the normalised gradient, extended to
 *     Phong (ambient + clamped diffuse + specular).
 *   - Eq. 6 (§3.9) and §3.10 step 4: emission-absorption compositing, evaluated front to
 *     back with early ray termination.
 *
 * Readings taken where the paper is silent or garbled (each also listed in the design
 * notes of the repository):
 *   R1 world coordinates = voxel indices; s = raw / value_max.
 *   R2 camera: fwd = normalize(target-eye), right = normalize(fwd x up), up' = right x fwd;
 *      pixel centres u = (2(px+1/2)/W - 1) * ax, v = (1 - 2(py+1/2)/H) * ay with
 *      ay = tan(fov/2) (perspective) or ortho_height/2 (orthographic), ax = ay * W/H;
 *      perspective: o = eye, d = normalize(fwd + u right + v up'); orthographic:
 *      o = eye + u right + v up', d = fwd.  py = 0 is the top row.
 *   R3 the ray setup (basis, pixel rays, slab test, sample count K) decides integers,
 *      so it is evaluated in the paper's precision (FP32, OpenCL float4), with every
 *      operation rounded separately (this file is compiled with -ffp-contract=off);
 *      everything after it (sample positions, interpolation, shading, compositing) is FP64.
 *   R4 slab test; an axis with a zero direction component is inside iff lo <= o <= hi;
 *      the entry is clamped to t >= 0; K = floor((t_far - t_near)/step + 1/2) samples at
 *      t_k = t_near + (k + 1/2) step, k = 0..K-1.
 *   R5 trilinear interpolation of the clamp-to-edge extension E(j) = V(clamp(j, 0, n-1)):
 *      lerp along x, then y, then z.
 *   R6 transfer function: u = clamp(s (N-1), 0, N-1), i = min(floor(u), N-2), w = u - i,
 *      TF(s) = (1-w) T[i] + w T[i+1] on all four channels; no opacity correction for the
 *      step size.
 *   R7 every gradient tap is E-trilinear at p + offset (clamp-to-edge addressing);
 *      Sobel3D: all three components are the x mask rotated onto their axis, + on the
 *      +1 side (the printed y/z masks are garbled); Zucker-Hummel: weight of neighbour
 *      (+-1, b, c) is +-1/sqrt(1 + b^2 + c^2); result scaled by 1/(2 S_side) with S_side
 *      the sum of one side's weights (1, 22, 1 + 4/sqrt2 + 4/sqrt3).
 *   R8 N = -g/|g| if |g| > 1e-6 else 0 (points towards lower values: outward normal);
 *      L = normalize(light - p) with light = eye for a headlight; V = -d (orthographic)
 *      or normalize(eye - p) (perspective); diff = max(0, N.L); spec = (N.L > 0) ?
 *      max(0, R.V)^shininess : 0 with R = 2 (N.L) N - L; c = rgb (ka + kd diff) + ks spec.
 *   R9 front to back: C += T a c, T *= (1 - a); stop after the sample where 1 - T >= ert
 *      (§3.9's end of the recursion at zero alpha read as transmittance -> 0).  Output (C, 1 - T),
 *      premultiplied over black.  Shading is skipped where a == 0 (it adds nothing).
 *
 *   R16 adaptive sampling (§5.2: coarser sampling in detail-poor regions): the regions are
 *      32^3-voxel blocks; a region whose footprint [32r - 1, 32r + 33] (clipped to the
 *      volume) has a value range max - min (raw units, FP32) <= adapt_range4 has multiplier
 *      m = 4, else <= adapt_range2 m = 2, else m = 1 (a negative bound disables its level).
 *      Sample k of R4 is taken iff k mod m(region(p_k)) == 0, with the region of its FP32
 *      position (R13's FP32 position, floor >> 5, clamped to the region grid), and stands
 *      for m samples: its opacity is corrected to 1 - (1 - a)^m.  With every m = 1 this is
 *      R4-R9 unchanged.
 *
 * First-hit surfaces (the renderer the paper itself implements, §3.11, with the hitpoint
 * refinement of §5.1):
 *   R13 a threshold window [lo, hi] of raw voxel values marks solid matter; the coarse
 *      samples are the samples of R4 with the coarse step; the first one inside the window
 *      is the hit.  The inside tests decide integers and branches, so they are evaluated in
 *      FP32 (the paper's precision) as: t_k = fma(k + 1/2, step, t_near),
 *      p = fma(t, d, o) per axis, i0 = clamp(floor(p), 0, n - 2), f = p - i0, trilinear of
 *      the raw values with lerps fma(f, b - a, a) along x, then y, then z; inside iff
 *      lo <= s <= hi.
 *   R14 refinement (§5.1: step back half a step, then halve the step, moving back while
 *      inside and forward while outside, 5-6 times) = bisection of [a, b] = [t_{k-1}, t_k]
 *      ([t_near, t_0] for k = 0) keeping a outside and b inside, m = (a + b) * 1/2 in FP32,
 *      `refine` steps; the hit is the midpoint of the final bracket.  If k = 0 and the
 *      entry point itself is inside, the hit is the entry point.
 *   R15 at the hit point p = o + t d (FP64 from here on): N = -g/|g| (R7, R8) turned to face
 *      the viewer (N.d <= 0, so surfaces entered from either side of the window are lit);
 *      L, V and Phong as R8 with the surface colour; output (c, 1) and the depth t; a ray
 *      without a hit gives (0, 0, 0, 0) and depth +inf.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { VRO_GRAD_CENTRAL = 0, VRO_GRAD_SOBEL3D = 1, VRO_GRAD_ZUCKER_HUMMEL = 2 };
enum { VRO_U8 = 0, VRO_U16 = 1, VRO_F32 = 2, VRO_F64 = 3 };

typedef struct {
    float eye[3], target[3], up[3];
    int ortho;
    float fov_y_deg, ortho_height;
    int width, height;
} vro_camera;

typedef struct {
    float step;
    int grad;
    double ka, kd, ks, shininess;
    double light[3];
    int headlight;
    double ert_threshold;
    float clip_lo[3], clip_hi[3];
    double adapt_range2, adapt_range4; /* R16 adaptive sampling; negative = off */
} vro_params;

typedef struct {
    const void *data; /* raw voxels, x fastest: index x + nx*(y + ny*z) */
    int dtype;
    int n[3];
    double value_max;
} vro_volume;

/* ------------------------------------------------------------------ voxel access */
static double raw_at(const vro_volume *vol, long idx)
{
    switch (vol->dtype) {
    case VRO_U8: return (double)((const uint8_t *)vol->data)[idx];
    case VRO_U16: return (double)((const uint16_t *)vol->data)[idx];
    case VRO_F32: return (double)((const float *)vol->data)[idx];
    default: return ((const double *)vol->data)[idx];
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* E(j): the clamp-to-edge extension of the volume (reading R5), normalised (R1). */
static double E(const vro_volume *vol, int x, int y, int z)
{
    x = clampi(x, 0, vol->n[0] - 1);
    y = clampi(y, 0, vol->n[1] - 1);
    z = clampi(z, 0, vol->n[2] - 1);
    long idx = (long)x + (long)vol->n[0] * ((long)y + (long)vol->n[1] * (long)z);
    return raw_at(vol, idx) / vol->value_max;
}

/* Eq. 2: g(x) = f(x0) + (f(x1) - f(x0)) / (x1 - x0) * (x - x0), with x1 - x0 = 1. */
static double lerp(double f0, double f1, double t) { return f0 + (f1 - f0) * t; }

/* §3.4: trilinear interpolation = four lerps along x, two along y, one along z. */
double vro_sample(const vro_volume *vol, const double p[3])
{
    int i[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        i[a] = (int)fl;
        f[a] = p[a] - fl;
    }
    double c000 = E(vol, i[0], i[1], i[2]), c100 = E(vol, i[0] + 1, i[1], i[2]);
    double c010 = E(vol, i[0], i[1] + 1, i[2]), c110 = E(vol, i[0] + 1, i[1] + 1, i[2]);
    double c001 = E(vol, i[0], i[1], i[2] + 1), c101 = E(vol, i[0] + 1, i[1], i[2] + 1);
    double c011 = E(vol, i[0], i[1] + 1, i[2] + 1), c111 = E(vol, i[0] + 1, i[1] + 1, i[2] + 1);
    double x00 = lerp(c000, c100, f[0]), x10 = lerp(c010, c110, f[0]);
    double x01 = lerp(c001, c101, f[0]), x11 = lerp(c011, c111, f[0]);
    double y0 = lerp(x00, x10, f[1]), y1 = lerp(x01, x11, f[1]);
    return lerp(y0, y1, f[2]);
}

/* Trilinear corner weights and indices of E at p (used by the adjoint). */
static void trilinear_corners(const double p[3], int base[3], double w[8])
{
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        base[a] = (int)fl;
        f[a] = p[a] - fl;
    }
    for (int c = 0; c < 8; ++c) {
        double wx = (c & 1) ? f[0] : 1.0 - f[0];
        double wy = (c & 2) ? f[1] : 1.0 - f[1];
        double wz = (c & 4) ? f[2] : 1.0 - f[2];
        w[c] = wx * wy * wz;
    }
}

/* ---------------------------------------------------------- gradient operators */
/* Tap list of one gradient component along axis `ax`: offsets and weights.
 * Returns the number of taps and the scale 1/(2 S_side) (reading R7). */
static int operator_taps(int op, int ax, int off[54][3], double wt[54], double *scale)
{
    int n = 0;
    int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
    if (op == VRO_GRAD_CENTRAL) {
        /* Eq. 3: delta = V(P + e) - V(P - e). */
        for (int side = -1; side <= 1; side += 2) {
            off[n][0] = off[n][1] = off[n][2] = 0;
            off[n][ax] = side;
            wt[n] = (double)side;
            ++n;
        }
        *scale = 1.0 / 2.0;
        return n;
    }
    double s_side = 0.0;
    for (int side = -1; side <= 1; side += 2) {
        for (int b = -1; b <= 1; ++b) {
            for (int c = -1; c <= 1; ++c) {
                double w;
                if (op == VRO_GRAD_SOBEL3D) {
                    /* Eq. 4: plane weights [[1,3,1],[3,6,3],[1,3,1]]. */
                    static const double sob[3][3] = {{1, 3, 1}, {3, 6, 3}, {1, 3, 1}};
                    w = sob[b + 1][c + 1];
                } else {
                    /* Zucker-Hummel: direction cosine of the neighbour (+-1, b, c). */
                    w = 1.0 / sqrt(1.0 + (double)(b * b) + (double)(c * c));
                }
                off[n][ax] = side;
                off[n][o1] = b;
                off[n][o2] = c;
                wt[n] = side * w;
                if (side == 1) s_side += w;
                ++n;
            }
        }
    }
    *scale = 1.0 / (2.0 * s_side);
    return n;
}

/* Scaled gradient estimate g_hat at p (reading R7): each tap is E-trilinear at p + off. */
void vro_gradient(const vro_volume *vol, int op, const double p[3], double g[3])
{
    int off[54][3];
    double wt[54], scale;
    for (int ax = 0; ax < 3; ++ax) {
        int n = operator_taps(op, ax, off, wt, &scale);
        double acc = 0.0;
        for (int t = 0; t < n; ++t) {
            double q[3] = {p[0] + off[t][0], p[1] + off[t][1], p[2] + off[t][2]};
            acc += wt[t] * vro_sample(vol, q);
        }
        g[ax] = acc * scale;
    }
}

/* ------------------------------------------------------------- transfer function */
/* §3.7 lookup table, read with linear interpolation between entries (reading R6).
 * dslope (optional) receives d(rgba)/ds. */
void vro_tf(const double *tf, int n, double s, double out[4], double dslope[4])
{
    double u = s * (double)(n - 1);
    int inside = 1;
    if (u < 0.0) { u = 0.0; inside = 0; }
    if (u > (double)(n - 1)) { u = (double)(n - 1); inside = 0; }
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    double w = u - (double)i;
    for (int c = 0; c < 4; ++c) {
        out[c] = (1.0 - w) * tf[4 * i + c] + w * tf[4 * (i + 1) + c];
        if (dslope) dslope[c] = inside ? (tf[4 * (i + 1) + c] - tf[4 * i + c]) * (double)(n - 1) : 0.0;
    }
}

/* ---------------------------------------------------------------------- shading */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normalize3(const double v[3], double out[3])
{
    double l = sqrt(dot3(v, v));
    for (int a = 0; a < 3; ++a) out[a] = l > 0.0 ? v[a] / l : 0.0;
}

/* Listing 3 ("Volume Shading") extended to Phong (reading R8). */
void vro_shade(const double N[3], const double L[3], const double V[3], const double rgb[3],
               double ka, double kd, double ks, double shininess, double c[3])
{
    double nl = dot3(N, L);
    double diff = nl > 0.0 ? nl : 0.0;
    double spec = 0.0;
    if (nl > 0.0) {
        double R[3];
        for (int a = 0; a < 3; ++a) R[a] = 2.0 * nl * N[a] - L[a];
        double rv = dot3(R, V);
        spec = rv > 0.0 ? pow(rv, shininess) : 0.0;
    }
    for (int a = 0; a < 3; ++a) c[a] = rgb[a] * (ka + kd * diff) + ks * spec;
}

/* Outward unit normal from the gradient estimate (reading R8). */
static void normal_from_gradient(const double g[3], double N[3], double *gnorm)
{
    double l = sqrt(dot3(g, g));
    *gnorm = l;
    for (int a = 0; a < 3; ++a) N[a] = l > 1e-6 ? -g[a] / l : 0.0;
}

/* ------------------------------------------------------------------ compositing */
/* Eq. 6 front to back with early termination (reading R9) over a given sample sequence.
 * Returns the number of samples consumed. */
int vro_composite(const double *alpha, const double *rgb, int n, double ert, double out[4])
{
    double C[3] = {0, 0, 0}, T = 1.0;
    int k;
    for (k = 0; k < n; ++k) {
        for (int a = 0; a < 3; ++a) C[a] += T * alpha[k] * rgb[3 * k + a];
        T *= 1.0 - alpha[k];
        if (1.0 - T >= ert) { ++k; break; }
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    return k;
}

/* ----------------------------------------------------------- FP32 ray setup (R3) */
static float f_dot3(const float a[3], const float b[3])
{
    float r = a[0] * b[0];
    r = r + a[1] * b[1];
    r = r + a[2] * b[2];
    return r;
}

static void f_normalize(float v[3])
{
    float l = sqrtf(f_dot3(v, v));
    v[0] = v[0] / l;
    v[1] = v[1] / l;
    v[2] = v[2] / l;
}

static void f_cross(const float a[3], const float b[3], float r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

typedef struct {
    float eye[3], fwd[3], right[3], upv[3];
    float ax, ay;
    int ortho, width, height;
} vro_basis;

static void camera_basis(const vro_camera *cam, vro_basis *b)
{
    for (int a = 0; a < 3; ++a) {
        b->eye[a] = cam->eye[a];
        b->fwd[a] = cam->target[a] - cam->eye[a];
    }
    f_normalize(b->fwd);
    f_cross(b->fwd, cam->up, b->right);
    f_normalize(b->right);
    f_cross(b->right, b->fwd, b->upv);
    double half;
    if (cam->ortho) half = (double)(cam->ortho_height / 2.0f);
    else half = tan(((double)cam->fov_y_deg * M_PI) / 360.0);
    b->ay = (float)half;
    b->ax = (float)((half * (double)cam->width) / (double)cam->height);
    b->ortho = cam->ortho;
    b->width = cam->width;
    b->height = cam->height;
}

/* Box = clip box intersected with the volume box [0, n-1] (§3.6). */
static void render_box(const vro_params *prm, const int n[3], float lo[3], float hi[3])
{
    for (int a = 0; a < 3; ++a) {
        float vhi = (float)(n[a] - 1);
        lo[a] = prm->clip_lo[a] > 0.0f ? prm->clip_lo[a] : 0.0f;
        hi[a] = prm->clip_hi[a] < vhi ? prm->clip_hi[a] : vhi;
    }
}

/* Ray of pixel (px, py) and its sample count.  Returns 1 on a hit (K may still be 0). */
static int ray_setup(const vro_basis *b, const float lo[3], const float hi[3], float step,
                     int px, int py, float o[3], float d[3], float *t_near, int *K)
{
    float sx = (float)(2 * px + 1) / (float)b->width - 1.0f;
    float sy = 1.0f - (float)(2 * py + 1) / (float)b->height;
    float u = sx * b->ax, v = sy * b->ay;
    if (b->ortho) {
        for (int a = 0; a < 3; ++a) {
            float t = b->eye[a] + u * b->right[a];
            o[a] = t + v * b->upv[a];
            d[a] = b->fwd[a];
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            float t = b->fwd[a] + u * b->right[a];
            d[a] = t + v * b->upv[a];
            o[a] = b->eye[a];
        }
        f_normalize(d);
    }
    float tn = 0.0f, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (lo[a] > hi[a]) { *K = 0; *t_near = 0.0f; return 0; }
        if (d[a] == 0.0f) {
            if (o[a] < lo[a] || o[a] > hi[a]) { *K = 0; *t_near = 0.0f; return 0; }
        } else {
            float t0 = (lo[a] - o[a]) / d[a];
            float t1 = (hi[a] - o[a]) / d[a];
            float tmin = t0 < t1 ? t0 : t1, tmax = t0 < t1 ? t1 : t0;
            if (tmin > tn) tn = tmin;
            if (tmax < tf) tf = tmax;
        }
    }
    *t_near = tn;
    if (!(tf >= tn)) { *K = 0; return 0; }
    float kf = floorf((tf - tn) / step + 0.5f);
    *K = kf > 0.0f ? (int)kf : 0;
    return 1;
}

/* Test hook: the FP32 ray of one pixel. */
int vro_ray(const vro_camera *cam, const vro_params *prm, const int n[3], int px, int py,
            float o[3], float d[3], float *t_near, int *K)
{
    vro_basis b;
    float lo[3], hi[3];
    camera_basis(cam, &b);
    render_box(prm, n, lo, hi);
    return ray_setup(&b, lo, hi, prm->step, px, py, o, d, t_near, K);
}

/* ------------------------------------------------------------------ one ray */
typedef struct {
    double p[3], s, rgba[4], dslope[4], g[3], gnorm, N[3], L[3], V[3], c[3], T;
} vro_sample_rec;

static void sample_point(const float o[3], const float d[3], float t_near, float step, int k,
                         double p[3])
{
    double t = (double)t_near + ((double)k + 0.5) * (double)step;
    for (int a = 0; a < 3; ++a) p[a] = (double)o[a] + t * (double)d[a];
}

static void light_view(const vro_basis *b, const vro_params *prm, const float d[3],
                       const double p[3], double L[3], double V[3])
{
    double lp[3], lv[3], ev[3];
    for (int a = 0; a < 3; ++a) lp[a] = prm->headlight ? (double)b->eye[a] : prm->light[a];
    for (int a = 0; a < 3; ++a) lv[a] = lp[a] - p[a];
    normalize3(lv, L);
    if (b->ortho) {
        for (int a = 0; a < 3; ++a) V[a] = -(double)d[a];
    } else {
        for (int a = 0; a < 3; ++a) ev[a] = (double)b->eye[a] - p[a];
        normalize3(ev, V);
    }
}

/* Evaluate sample k fully (value, TF, gradient, normal, shading), as §3.10 steps 2-3. */
static void eval_sample(const vro_volume *vol, const double *tf, int ntf, const vro_basis *b,
                        const vro_params *prm, const float o[3], const float d[3], float t_near,
                        int k, vro_sample_rec *r)
{
    sample_point(o, d, t_near, prm->step, k, r->p);
    r->s = vro_sample(vol, r->p);
    vro_tf(tf, ntf, r->s, r->rgba, r->dslope);
    vro_gradient(vol, prm->grad, r->p, r->g);
    normal_from_gradient(r->g, r->N, &r->gnorm);
    light_view(b, prm, d, r->p, r->L, r->V);
    vro_shade(r->N, r->L, r->V, r->rgba, prm->ka, prm->kd, prm->ks, prm->shininess, r->c);
}

/* ------------------------------------------------------------ adaptive sampling (R16) */
enum { VRO_REGION = 32, VRO_REGION_SHIFT = 5 };
static int brick_count(int n) { return (n + VRO_REGION - 1) / VRO_REGION; }

/* Multiplier of every region (NULL when adaptive sampling is off), from the raw value range
 * of its footprint [32r - 1, 32r + 33] clipped to the volume. */
static unsigned char *brick_multipliers(const vro_volume *vol, const vro_params *prm)
{
    if (prm->adapt_range2 < 0.0 && prm->adapt_range4 < 0.0) return NULL;
    int nb[3] = {brick_count(vol->n[0]), brick_count(vol->n[1]), brick_count(vol->n[2])};
    unsigned char *m = (unsigned char *)malloc((size_t)nb[0] * nb[1] * nb[2]);
    for (int bz = 0; bz < nb[2]; ++bz)
        for (int by = 0; by < nb[1]; ++by)
            for (int bx = 0; bx < nb[0]; ++bx) {
                int b[3] = {bx, by, bz}, lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = clampi(VRO_REGION * b[a] - 1, 0, vol->n[a] - 1);
                    hi[a] = clampi(VRO_REGION * b[a] + VRO_REGION + 1, 0, vol->n[a] - 1);
                }
                double mn = INFINITY, mx = -INFINITY;
                for (int z = lo[2]; z <= hi[2]; ++z)
                    for (int y = lo[1]; y <= hi[1]; ++y)
                        for (int x = lo[0]; x <= hi[0]; ++x) {
                            double v = raw_at(vol, (long)x + (long)vol->n[0] * ((long)y + (long)vol->n[1] * z));
                            if (v < mn) mn = v;
                            if (v > mx) mx = v;
                        }
                float range = (float)mx - (float)mn;
                int mult = 1;
                if (prm->adapt_range4 >= 0.0 && range <= (float)prm->adapt_range4) mult = 4;
                else if (prm->adapt_range2 >= 0.0 && range <= (float)prm->adapt_range2) mult = 2;
                m[bx + nb[0] * (by + nb[1] * bz)] = (unsigned char)mult;
            }
    return m;
}

/* Multiplier of sample k of the ray (o, d, t_near): region of its FP32 position. */
static int sample_multiplier(const vro_volume *vol, const unsigned char *mult, const float o[3],
                             const float d[3], float t_near, float step, int k)
{
    float t = fmaf((float)k + 0.5f, step, t_near);
    int b[3];
    for (int a = 0; a < 3; ++a) {
        float p = fmaf(t, d[a], o[a]);
        b[a] = clampi(((int)floorf(p)) >> VRO_REGION_SHIFT, 0, brick_count(vol->n[a]) - 1);
    }
    return mult[b[0] + brick_count(vol->n[0]) * (b[1] + brick_count(vol->n[1]) * b[2])];
}

/* Render one pixel; returns the samples marched (the plain method's count). */
static int render_pixel(const vro_volume *vol, const double *tf, int ntf, const vro_basis *b,
                        const float lo[3], const float hi[3], const vro_params *prm,
                        const unsigned char *mult, int px, int py, double out[4])
{
    float o[3], d[3], tn;
    int K;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (!ray_setup(b, lo, hi, prm->step, px, py, o, d, &tn, &K)) return 0;
    double C[3] = {0, 0, 0}, T = 1.0;
    int k;
    for (k = 0; k < K; ++k) {
        int m = 1;
        if (mult) {
            m = sample_multiplier(vol, mult, o, d, tn, prm->step, k);
            if (k % m != 0) continue; /* not on this region's coarser grid */
        }
        double p[3], rgba[4];
        sample_point(o, d, tn, prm->step, k, p);
        double s = vro_sample(vol, p);
        vro_tf(tf, ntf, s, rgba, NULL);
        double alpha = m == 1 ? rgba[3] : 1.0 - pow(1.0 - rgba[3], (double)m);
        if (alpha != 0.0) {
            double g[3], N[3], L[3], V[3], c[3], gn;
            vro_gradient(vol, prm->grad, p, g);
            normal_from_gradient(g, N, &gn);
            light_view(b, prm, d, p, L, V);
            vro_shade(N, L, V, rgba, prm->ka, prm->kd, prm->ks, prm->shininess, c);
            for (int a = 0; a < 3; ++a) C[a] += T * alpha * c[a];
            T *= 1.0 - alpha;
        }
        if (1.0 - T >= prm->ert_threshold) { ++k; break; }
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    return k;
}

/* Render rows [row0, row1) of the image into out_rgba (H x W x 4, row-major, only those
 * rows written).  counts (optional, H x W) receives the samples marched per ray.
 * Returns the total sample count of the rendered rows. */
long long vro_render(const vro_volume *vol, const double *tf, int ntf, const vro_camera *cam,
                     const vro_params *prm, double *out_rgba, int *counts, int row0, int row1,
                     int nthreads)
{
    vro_basis b;
    float lo[3], hi[3];
    camera_basis(cam, &b);
    render_box(prm, vol->n, lo, hi);
    long long total = 0;
    int W = cam->width;
    unsigned char *mult = brick_multipliers(vol, prm);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
#endif
    for (int py = row0; py < row1; ++py) {
        for (int px = 0; px < W; ++px) {
            long pix = (long)py * W + px;
            int k = render_pixel(vol, tf, ntf, &b, lo, hi, prm, mult, px, py, out_rgba + 4 * pix);
            if (counts) counts[pix] = k;
            total += k;
        }
    }
    free(mult);
    return total;
}

/* Render an explicit list of pixels (for sampled comparisons at full size). */
long long vro_render_pixels(const vro_volume *vol, const double *tf, int ntf,
                            const vro_camera *cam, const vro_params *prm, const int *px,
                            const int *py, int npix, double *out_rgba, int *counts, int nthreads)
{
    vro_basis b;
    float lo[3], hi[3];
    camera_basis(cam, &b);
    render_box(prm, vol->n, lo, hi);
    long long total = 0;
    unsigned char *mult = brick_multipliers(vol, prm);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
#endif
    for (int i = 0; i < npix; ++i) {
        int k = render_pixel(vol, tf, ntf, &b, lo, hi, prm, mult, px[i], py[i],
                             out_rgba + 4 * (long)i);
        if (counts) counts[i] = k;
        total += k;
    }
    free(mult);
    return total;
}

/* ------------------------------------------------------------ first-hit surfaces */
typedef struct {
    float step, iso_lo, iso_hi;
    int refine, grad;
    double ka, kd, ks, shininess;
    double light[3];
    int headlight;
    double color[3];
    float clip_lo[3], clip_hi[3];
} vro_surface_params;

/* Raw voxel value at the clamp-to-edge position, as FP32. */
static float raw_f32(const vro_volume *vol, int x, int y, int z)
{
    x = clampi(x, 0, vol->n[0] - 1);
    y = clampi(y, 0, vol->n[1] - 1);
    z = clampi(z, 0, vol->n[2] - 1);
    return (float)raw_at(vol, (long)x + (long)vol->n[0] * ((long)y + (long)vol->n[1] * (long)z));
}

static float lerp_f32(float a, float b, float f) { return fmaf(f, b - a, a); }

/* Reading R13: the FP32 trilinear value (raw units) that decides inside / outside. */
float vro_sample_f32(const vro_volume *vol, const float p[3])
{
    int i[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
        int top = vol->n[a] > 1 ? vol->n[a] - 2 : 0;
        i[a] = clampi((int)floorf(p[a]), 0, top);
        f[a] = p[a] - (float)i[a];
    }
    float c000 = raw_f32(vol, i[0], i[1], i[2]), c100 = raw_f32(vol, i[0] + 1, i[1], i[2]);
    float c010 = raw_f32(vol, i[0], i[1] + 1, i[2]), c110 = raw_f32(vol, i[0] + 1, i[1] + 1, i[2]);
    float c001 = raw_f32(vol, i[0], i[1], i[2] + 1), c101 = raw_f32(vol, i[0] + 1, i[1], i[2] + 1);
    float c011 = raw_f32(vol, i[0], i[1] + 1, i[2] + 1);
    float c111 = raw_f32(vol, i[0] + 1, i[1] + 1, i[2] + 1);
    float x00 = lerp_f32(c000, c100, f[0]), x10 = lerp_f32(c010, c110, f[0]);
    float x01 = lerp_f32(c001, c101, f[0]), x11 = lerp_f32(c011, c111, f[0]);
    float y0 = lerp_f32(x00, x10, f[1]), y1 = lerp_f32(x01, x11, f[1]);
    return lerp_f32(y0, y1, f[2]);
}

static int inside_at(const vro_volume *vol, const vro_surface_params *sp, const float o[3],
                     const float d[3], float t)
{
    float p[3];
    for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
    float s = vro_sample_f32(vol, p);
    return s >= sp->iso_lo && s <= sp->iso_hi;
}

/* One ray of the first-hit renderer (R13-R15).  Returns the coarse samples taken. */
static int surface_pixel(const vro_volume *vol, const vro_basis *b, const float lo[3],
                         const float hi[3], const vro_surface_params *sp, int px, int py,
                         double out[4], float *depth)
{
    float o[3], d[3], tn;
    int K;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    *depth = INFINITY;
    if (!ray_setup(b, lo, hi, sp->step, px, py, o, d, &tn, &K)) return 0;
    int k;
    for (k = 0; k < K; ++k)
        if (inside_at(vol, sp, o, d, fmaf((float)k + 0.5f, sp->step, tn))) break;
    if (k == K) return K;
    float t_hit;
    if (k == 0 && inside_at(vol, sp, o, d, tn)) {
        t_hit = tn;
    } else {
        float ta = k == 0 ? tn : fmaf((float)k - 0.5f, sp->step, tn);
        float tb = fmaf((float)k + 0.5f, sp->step, tn);
        for (int r = 0; r < sp->refine; ++r) {
            float m = 0.5f * (ta + tb);
            if (inside_at(vol, sp, o, d, m)) tb = m;
            else ta = m;
        }
        t_hit = 0.5f * (ta + tb);
    }
    *depth = t_hit;
    double p[3], g[3], N[3], gn, L[3], V[3], c[3], lp[3], lv[3], ev[3];
    for (int a = 0; a < 3; ++a) p[a] = (double)o[a] + (double)t_hit * (double)d[a];
    vro_gradient(vol, sp->grad, p, g);
    normal_from_gradient(g, N, &gn);
    if (N[0] * d[0] + N[1] * d[1] + N[2] * d[2] > 0.0)
        for (int a = 0; a < 3; ++a) N[a] = -N[a];
    for (int a = 0; a < 3; ++a) lp[a] = sp->headlight ? (double)b->eye[a] : sp->light[a];
    for (int a = 0; a < 3; ++a) lv[a] = lp[a] - p[a];
    normalize3(lv, L);
    if (b->ortho) {
        for (int a = 0; a < 3; ++a) V[a] = -(double)d[a];
    } else {
        for (int a = 0; a < 3; ++a) ev[a] = (double)b->eye[a] - p[a];
        normalize3(ev, V);
    }
    vro_shade(N, L, V, sp->color, sp->ka, sp->kd, sp->ks, sp->shininess, c);
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = 1.0;
    return k + 1;
}

/* Render rows [row0, row1) with the first-hit renderer; depth (H x W) receives the hit
 * distance along the unit ray (+inf where nothing is hit).  Returns the coarse samples. */
long long vro_render_surface(const vro_volume *vol, const vro_camera *cam,
                             const vro_surface_params *sp, double *out_rgba, float *depth,
                             int row0, int row1, int nthreads)
{
    vro_basis b;
    float lo[3], hi[3];
    vro_params box;
    camera_basis(cam, &b);
    for (int a = 0; a < 3; ++a) {
        box.clip_lo[a] = sp->clip_lo[a];
        box.clip_hi[a] = sp->clip_hi[a];
    }
    render_box(&box, vol->n, lo, hi);
    long long total = 0;
    int W = cam->width;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
#endif
    for (int py = row0; py < row1; ++py)
        for (int px = 0; px < W; ++px) {
            long pix = (long)py * W + px;
            total += surface_pixel(vol, &b, lo, hi, sp, px, py, out_rgba + 4 * pix, depth + pix);
        }
    return total;
}

int vro_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ reverse mode (FP64) */
/* Scatter dL/ds at point q (normalised units) onto the raw voxels: s = E-trilinear / vmax. */
static void scatter_sample(const vro_volume *vol, const double q[3], double ds, double *gvol)
{
    int base[3];
    double w[8];
    trilinear_corners(q, base, w);
    for (int c = 0; c < 8; ++c) {
        int x = clampi(base[0] + (c & 1), 0, vol->n[0] - 1);
        int y = clampi(base[1] + ((c >> 1) & 1), 0, vol->n[1] - 1);
        int z = clampi(base[2] + ((c >> 2) & 1), 0, vol->n[2] - 1);
        long idx = (long)x + (long)vol->n[0] * ((long)y + (long)vol->n[1] * (long)z);
        gvol[idx] += w[c] * ds / vol->value_max;
    }
}

/* Straight-line reverse mode of render_pixel: every sample is stored, no checkpoints.
 * grad_rgba: dL/d(R,G,B,A) of this pixel.  Accumulates into gvol (raw-voxel units) and
 * gtf (ntf x 4). */
static void backward_pixel(const vro_volume *vol, const double *tf, int ntf, const vro_basis *b,
                           const float lo[3], const float hi[3], const vro_params *prm, int px,
                           int py, const double grad_rgba[4], double *gvol, double *gtf)
{
    float o[3], d[3], tn;
    int K;
    if (!ray_setup(b, lo, hi, prm->step, px, py, o, d, &tn, &K) || K == 0) return;
    vro_sample_rec *rec = (vro_sample_rec *)malloc(sizeof(vro_sample_rec) * (size_t)K);
    double T = 1.0;
    int kend = 0;
    for (int k = 0; k < K; ++k) {
        vro_sample_rec *r = &rec[k];
        eval_sample(vol, tf, ntf, b, prm, o, d, tn, k, r);
        r->T = T;
        kend = k + 1;
        if (r->rgba[3] != 0.0) T *= 1.0 - r->rgba[3];
        if (1.0 - T >= prm->ert_threshold) break;
    }
    const double *g = grad_rgba;
    double Tadj = -grad_rgba[3]; /* dL/dT_K, since A = 1 - T_K */
    for (int k = kend - 1; k >= 0; --k) {
        vro_sample_rec *r = &rec[k];
        double a = r->rgba[3];
        double gc = g[0] * r->c[0] + g[1] * r->c[1] + g[2] * r->c[2];
        double d_alpha = r->T * gc - r->T * Tadj;
        double dc[3];
        for (int q = 0; q < 3; ++q) dc[q] = r->T * a * g[q];
        Tadj = a * gc + (1.0 - a) * Tadj;
        /* shading: c = rgb (ka + kd diff) + ks spec */
        double nl = dot3(r->N, r->L);
        double diff = nl > 0.0 ? nl : 0.0;
        double drgba[4];
        for (int q = 0; q < 3; ++q) drgba[q] = dc[q] * (prm->ka + prm->kd * diff);
        drgba[3] = d_alpha;
        double d_diff = prm->kd * (dc[0] * r->rgba[0] + dc[1] * r->rgba[1] + dc[2] * r->rgba[2]);
        double d_spec = prm->ks * (dc[0] + dc[1] + dc[2]);
        double dN[3] = {0, 0, 0};
        if (nl > 0.0) {
            for (int q = 0; q < 3; ++q) dN[q] += d_diff * r->L[q];
            double nv = dot3(r->N, r->V), lv = dot3(r->L, r->V);
            double x = 2.0 * nl * nv - lv; /* R.V */
            if (x > 0.0) {
                double dx = d_spec * prm->shininess * pow(x, prm->shininess - 1.0);
                for (int q = 0; q < 3; ++q) dN[q] += dx * (2.0 * nv * r->L[q] + 2.0 * nl * r->V[q]);
            }
        }
        /* normal: N = -g/|g| */
        if (r->gnorm > 1e-6) {
            double nh[3], dng = 0.0, dgv[3];
            for (int q = 0; q < 3; ++q) nh[q] = r->g[q] / r->gnorm;
            for (int q = 0; q < 3; ++q) dng += dN[q] * nh[q];
            for (int q = 0; q < 3; ++q) dgv[q] = -(dN[q] - dng * nh[q]) / r->gnorm;
            /* g_hat -> taps */
            int off[54][3];
            double wt[54], scale;
            for (int ax = 0; ax < 3; ++ax) {
                int nt = operator_taps(prm->grad, ax, off, wt, &scale);
                for (int t = 0; t < nt; ++t) {
                    double q3[3] = {r->p[0] + off[t][0], r->p[1] + off[t][1], r->p[2] + off[t][2]};
                    scatter_sample(vol, q3, wt[t] * scale * dgv[ax], gvol);
                }
            }
        }
        /* transfer function */
        double u = r->s * (double)(ntf - 1);
        if (u < 0.0) u = 0.0;
        if (u > (double)(ntf - 1)) u = (double)(ntf - 1);
        int i = (int)floor(u);
        if (i > ntf - 2) i = ntf - 2;
        double w = u - (double)i;
        double ds = 0.0;
        for (int q = 0; q < 4; ++q) {
            gtf[4 * i + q] += (1.0 - w) * drgba[q];
            gtf[4 * (i + 1) + q] += w * drgba[q];
            ds += drgba[q] * r->dslope[q];
        }
        scatter_sample(vol, r->p, ds, gvol);
    }
    free(rec);
}

/* Reverse mode over the whole image (serial: plain and obviously ordered). */
void vro_render_backward(const vro_volume *vol, const double *tf, int ntf, const vro_camera *cam,
                         const vro_params *prm, const double *grad_rgba, double *grad_vol,
                         double *grad_tf)
{
    vro_basis b;
    float lo[3], hi[3];
    camera_basis(cam, &b);
    render_box(prm, vol->n, lo, hi);
    for (int py = 0; py < cam->height; ++py)
        for (int px = 0; px < cam->width; ++px) {
            long pix = (long)py * cam->width + px;
            backward_pixel(vol, tf, ntf, &b, lo, hi, prm, px, py, grad_rgba + 4 * pix, grad_vol,
                           grad_tf);
        }
}
