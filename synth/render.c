/*
 * Seeded synthetic-scene renderer: ray casting of a textured sphere and/or
 * textured rectangles (a ground plane, fronto-parallel cards) into pinhole
 * images.
 *
 * This file is INPUT GENERATION only. It holds none of the photometric bundle
 * adjustment arithmetic (no warps of template pixels, no Jacobians, no
 * solves); it produces the images that both the CPU oracle and the GPU path
 * read. The scenes stand in for the paper's Blender-rendered sequence
 * (Sec. 4.1, "Synthetic Ground Truth"): an unlit (Lambertian-free, albedo
 * only) object so brightness constancy holds exactly between views.
 *
 * Albedo = fractal value noise on the 3-D surface point: `octaves` octaves,
 * frequency doubling and amplitude halving per octave, quintic fade
 * 6t^5-15t^4+10t^3, lattice values from the SplitMix64 mixing function of
 * Steele, Lea and Flood ("Fast splittable pseudorandom number generators",
 * OOPSLA 2014), normalised by the amplitude sum so values lie in [0,1).
 *
 * Camera convention: x right, y down, z forward; world point X maps to camera
 * coordinates R X + t with t = -R C.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static uint64_t splitmix64_mix(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform lattice value in [0,1) for integer cell corner (ix,iy,iz). */
static double lattice(int64_t ix, int64_t iy, int64_t iz, int octave, uint64_t seed)
{
    uint64_t h = splitmix64_mix(seed ^ (uint64_t)octave * 0xd1b54a32d192ed03ULL);
    h = splitmix64_mix(h ^ (uint64_t)ix);
    h = splitmix64_mix(h ^ (uint64_t)iy);
    h = splitmix64_mix(h ^ (uint64_t)iz);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

static double value_noise(double x, double y, double z, int octave, uint64_t seed)
{
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
    double sx = fade(x - fx), sy = fade(y - fy), sz = fade(z - fz);
    double c[2][2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                c[a][b][e] = lattice(ix + a, iy + b, iz + e, octave, seed);
    double x00 = c[0][0][0] + sx * (c[1][0][0] - c[0][0][0]);
    double x10 = c[0][1][0] + sx * (c[1][1][0] - c[0][1][0]);
    double x01 = c[0][0][1] + sx * (c[1][0][1] - c[0][0][1]);
    double x11 = c[0][1][1] + sx * (c[1][1][1] - c[0][1][1]);
    double y0 = x00 + sy * (x10 - x00);
    double y1 = x01 + sy * (x11 - x01);
    return y0 + sz * (y1 - y0);
}

/* Fractal value-noise albedo in [0,1). */
double synth_albedo(double x, double y, double z, double base_freq, int octaves, uint64_t seed)
{
    double sum = 0.0, amp = 1.0, norm = 0.0, freq = base_freq;
    for (int o = 0; o < octaves; ++o) {
        sum += amp * value_noise(x * freq, y * freq, z * freq, o, seed);
        norm += amp;
        amp *= 0.5;
        freq *= 2.0;
    }
    return sum / norm;
}

/* Scene: optional sphere at the origin plus rectangles. A rectangle row of
 * `rects` holds centre(3), unit axis a(3), unit axis b(3), half sizes ha, hb
 * (11 doubles); its plane has normal a x b. The ground plane of the larger
 * scenes is one such rectangle. */
typedef struct {
    double sphere_r;        /* <= 0: no sphere */
    int n_rects;
    const double* rects;
} scene_t;

/* Nearest positive ray parameter s along C + s*d that hits the scene.
 * Returns 0 for no hit, 1 for the sphere, 2 + i for rectangle i. */
static int cast(const scene_t* sc, const double C[3], const double d[3], double* s_out)
{
    int obj = 0;
    double best = INFINITY;
    if (sc->sphere_r > 0.0) {
        double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double b = C[0] * d[0] + C[1] * d[1] + C[2] * d[2];
        double c = C[0] * C[0] + C[1] * C[1] + C[2] * C[2] - sc->sphere_r * sc->sphere_r;
        double disc = b * b - a * c;
        if (disc >= 0.0) {
            double s = (-b - sqrt(disc)) / a;
            if (s > 1e-9 && s < best) { best = s; obj = 1; }
        }
    }
    for (int i = 0; i < sc->n_rects; ++i) {
        const double* r = sc->rects + 11 * i;
        const double *c0 = r, *ea = r + 3, *eb = r + 6;
        double nrm[3] = {ea[1] * eb[2] - ea[2] * eb[1], ea[2] * eb[0] - ea[0] * eb[2],
                         ea[0] * eb[1] - ea[1] * eb[0]};
        double den = nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2];
        if (fabs(den) < 1e-12) continue;
        double s = (nrm[0] * (c0[0] - C[0]) + nrm[1] * (c0[1] - C[1]) + nrm[2] * (c0[2] - C[2])) / den;
        if (!(s > 1e-9 && s < best)) continue;
        double P[3] = {C[0] + s * d[0] - c0[0], C[1] + s * d[1] - c0[1], C[2] + s * d[2] - c0[2]};
        double pa = P[0] * ea[0] + P[1] * ea[1] + P[2] * ea[2];
        double pb = P[0] * eb[0] + P[1] * eb[1] + P[2] * eb[2];
        if (fabs(pa) <= r[9] && fabs(pb) <= r[10]) { best = s; obj = 2 + i; }
    }
    *s_out = best;
    return obj;
}

/*
 * Render one H x W image with ss x ss supersampling (box filter over the
 * pixel footprint; sample (i,j) of pixel (u,v) sits at u-0.5+(i+0.5)/ss).
 * out[v*W+u] receives the mean albedo (background where a sample misses).
 * hit (nullable) receives per pixel the object id seen by every sample
 * (1 sphere, 2+i rectangle i), 0 when the samples see background, and 255
 * when they see more than one thing.
 */
void synth_render(int W, int H, int ss, double fx, double fy, double cx, double cy,
                  const double* R, const double* C, double sphere_r, int n_rects,
                  const double* rects, double base_freq, int octaves,
                  uint64_t seed, double background, float* out, unsigned char* hit)
{
    scene_t sc = {sphere_r, n_rects, rects};
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            double acc = 0.0;
            int first = -1, mixed = 0;
            for (int j = 0; j < ss; ++j) {
                for (int i = 0; i < ss; ++i) {
                    double pu = u - 0.5 + (i + 0.5) / ss;
                    double pv = v - 0.5 + (j + 0.5) / ss;
                    double dc[3] = {(pu - cx) / fx, (pv - cy) / fy, 1.0};
                    /* camera -> world direction: R^T dc */
                    double d[3];
                    for (int k = 0; k < 3; ++k)
                        d[k] = R[0 * 3 + k] * dc[0] + R[1 * 3 + k] * dc[1] + R[2 * 3 + k] * dc[2];
                    double s;
                    int obj = cast(&sc, C, d, &s);
                    if (first < 0) first = obj;
                    else if (obj != first) mixed = 1;
                    if (obj == 0) {
                        acc += background;
                    } else {
                        double X = C[0] + s * d[0], Y = C[1] + s * d[1], Z = C[2] + s * d[2];
                        acc += synth_albedo(X, Y, Z, base_freq, octaves, seed);
                    }
                }
            }
            out[(size_t)v * W + u] = (float)(acc / (ss * ss));
            if (hit) hit[(size_t)v * W + u] = mixed ? 255 : (unsigned char)first;
        }
    }
}

/* Cast rays through pixel centres (u,v) of a camera; returns the hit object
 * per ray and the world hit point (for ground-truth depths of points). */
void synth_cast_pixels(int n, const double* uv, double fx, double fy, double cx, double cy,
                       const double* R, const double* C, double sphere_r, int n_rects,
                       const double* rects, int* obj_out, double* X_out)
{
    scene_t sc = {sphere_r, n_rects, rects};
    for (int p = 0; p < n; ++p) {
        double dc[3] = {(uv[2 * p] - cx) / fx, (uv[2 * p + 1] - cy) / fy, 1.0};
        double d[3];
        for (int k = 0; k < 3; ++k)
            d[k] = R[0 * 3 + k] * dc[0] + R[1 * 3 + k] * dc[1] + R[2 * 3 + k] * dc[2];
        double s;
        int obj = cast(&sc, C, d, &s);
        obj_out[p] = obj;
        for (int k = 0; k < 3; ++k) X_out[3 * p + k] = obj ? C[k] + s * d[k] : NAN;
    }
}

/* First hit along the segment from camera centre C to world point X:
 * returns 1 when nothing blocks X (within a relative tolerance). */
void synth_unoccluded(int n, const double* X, const double* C, double sphere_r, int n_rects,
                      const double* rects, unsigned char* out)
{
    scene_t sc = {sphere_r, n_rects, rects};
    for (int p = 0; p < n; ++p) {
        double d[3] = {X[3 * p] - C[0], X[3 * p + 1] - C[1], X[3 * p + 2] - C[2]};
        double s;
        int obj = cast(&sc, C, d, &s);
        out[p] = (obj != 0 && s > 1.0 - 1e-7) || obj == 0;
    }
}
