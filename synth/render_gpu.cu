/*
 * Seeded synthetic-scene renderer on the GPU: the ray caster of render.c
 * (textured sphere and rectangles, fractal value-noise albedo, ss x ss box
 * supersampling) with one thread per pixel and every frame of a bundle in
 * one launch.
 *
 * INPUT GENERATION only, like render.c: no photometric bundle adjustment
 * arithmetic. The operations are the host renderer's, in its order, in
 * FP64, and the file is compiled without multiply-add contraction (as is
 * render.c), so both produce the same images bit for bit: double division
 * and square root are correctly rounded on either side, floor is exact and
 * the lattice hash is integer arithmetic.
 *
 * Lattice values: SplitMix64's mixing function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) chained
 * over (octave, ix, iy, iz); the chain prefixes shared by the eight corners
 * of a cell are mixed once (15 mixes per cell instead of 32, the same
 * values).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#define SYNTH_MAX_RECTS 8

struct SceneParams {
    double fx, fy, cx, cy, sphere_r, base_freq, background;
    unsigned long long seed;
    int W, H, ss, octaves, n_rects, F;
    double rects[SYNTH_MAX_RECTS * 11];
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

__device__ __forceinline__ double unit(unsigned long long h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

__device__ double value_noise(double x, double y, double z, int octave, unsigned long long seed)
{
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const long long ix = (long long)fx, iy = (long long)fy, iz = (long long)fz;
    const double sx = fade(x - fx), sy = fade(y - fy), sz = fade(z - fz);
    const unsigned long long h0 = mix64(seed ^ (unsigned long long)octave * 0xd1b54a32d192ed03ULL);
    double c[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const unsigned long long ha = mix64(h0 ^ (unsigned long long)(ix + a));
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const unsigned long long hb = mix64(ha ^ (unsigned long long)(iy + b));
#pragma unroll
            for (int e = 0; e < 2; ++e) c[a][b][e] = unit(mix64(hb ^ (unsigned long long)(iz + e)));
        }
    }
    const double x00 = c[0][0][0] + sx * (c[1][0][0] - c[0][0][0]);
    const double x10 = c[0][1][0] + sx * (c[1][1][0] - c[0][1][0]);
    const double x01 = c[0][0][1] + sx * (c[1][0][1] - c[0][0][1]);
    const double x11 = c[0][1][1] + sx * (c[1][1][1] - c[0][1][1]);
    const double y0 = x00 + sy * (x10 - x00);
    const double y1 = x01 + sy * (x11 - x01);
    return y0 + sz * (y1 - y0);
}

__device__ double albedo(double x, double y, double z, const SceneParams& p)
{
    double sum = 0.0, amp = 1.0, norm = 0.0, freq = p.base_freq;
    for (int o = 0; o < p.octaves; ++o) {
        sum += amp * value_noise(x * freq, y * freq, z * freq, o, p.seed);
        norm += amp;
        amp *= 0.5;
        freq *= 2.0;
    }
    return sum / norm;
}

/* nearest positive hit along C + s d: 0 none, 1 sphere, 2 + i rectangle i */
__device__ int cast(const SceneParams& p, const double* C, const double* d, double* s_out)
{
    int obj = 0;
    double best = __longlong_as_double(0x7ff0000000000000LL);
    if (p.sphere_r > 0.0) {
        const double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double b = C[0] * d[0] + C[1] * d[1] + C[2] * d[2];
        const double c = C[0] * C[0] + C[1] * C[1] + C[2] * C[2] - p.sphere_r * p.sphere_r;
        const double disc = b * b - a * c;
        if (disc >= 0.0) {
            const double s = (-b - sqrt(disc)) / a;
            if (s > 1e-9 && s < best) {
                best = s;
                obj = 1;
            }
        }
    }
    for (int i = 0; i < p.n_rects; ++i) {
        const double* r = p.rects + 11 * i;
        const double *c0 = r, *ea = r + 3, *eb = r + 6;
        const double nrm[3] = {ea[1] * eb[2] - ea[2] * eb[1], ea[2] * eb[0] - ea[0] * eb[2],
                               ea[0] * eb[1] - ea[1] * eb[0]};
        const double den = nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2];
        if (fabs(den) < 1e-12) continue;
        const double s = (nrm[0] * (c0[0] - C[0]) + nrm[1] * (c0[1] - C[1]) + nrm[2] * (c0[2] - C[2])) / den;
        if (!(s > 1e-9 && s < best)) continue;
        const double P[3] = {C[0] + s * d[0] - c0[0], C[1] + s * d[1] - c0[1], C[2] + s * d[2] - c0[2]};
        const double pa = P[0] * ea[0] + P[1] * ea[1] + P[2] * ea[2];
        const double pb = P[0] * eb[0] + P[1] * eb[1] + P[2] * eb[2];
        if (fabs(pa) <= r[9] && fabs(pb) <= r[10]) {
            best = s;
            obj = 2 + i;
        }
    }
    *s_out = best;
    return obj;
}

/* pixel (u, v) of frame blockIdx.z; RC: F x 12 (R row-major, then C) */
__global__ void __launch_bounds__(256) render_kernel(SceneParams p, const double* __restrict__ RC,
                                                     float* __restrict__ out, unsigned char* __restrict__ hit)
{
    const int u = blockIdx.x * 16 + (threadIdx.x & 15), v = blockIdx.y * 16 + (threadIdx.x >> 4);
    const int f = blockIdx.z;
    if (u >= p.W || v >= p.H) return;
    const double* R = RC + 12 * f;
    const double C[3] = {R[9], R[10], R[11]};
    double acc = 0.0;
    int first = -1, mixed = 0;
    for (int j = 0; j < p.ss; ++j) {
        for (int i = 0; i < p.ss; ++i) {
            const double pu = u - 0.5 + (i + 0.5) / p.ss;
            const double pv = v - 0.5 + (j + 0.5) / p.ss;
            const double dc[3] = {(pu - p.cx) / p.fx, (pv - p.cy) / p.fy, 1.0};
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = R[0 * 3 + k] * dc[0] + R[1 * 3 + k] * dc[1] + R[2 * 3 + k] * dc[2];
            double s;
            const int obj = cast(p, C, d, &s);
            if (first < 0) first = obj;
            else if (obj != first) mixed = 1;
            if (obj == 0) {
                acc += p.background;
            } else {
                const double X = C[0] + s * d[0], Y = C[1] + s * d[1], Z = C[2] + s * d[2];
                acc += albedo(X, Y, Z, p);
            }
        }
    }
    const size_t o = ((size_t)f * p.H + v) * p.W + u;
    out[o] = (float)(acc / (p.ss * p.ss));
    if (hit && f == 0) hit[(size_t)v * p.W + u] = mixed ? 255 : (unsigned char)first;
}

/*
 * Renders n_frames H x W images into out (device, frame-major), as
 * synth_render does frame by frame; hit (device, nullable) receives frame
 * 0's per-pixel object ids. RC: device, n_frames x 12 doubles (the
 * world-to-camera rotation row-major, then the camera centre). rects: host,
 * n_rects x 11 doubles (at most 8). Launches on the given stream; returns 0,
 * or a CUDA error code (1 for invalid arguments).
 */
extern "C" int synth_render_gpu(int n_frames, int W, int H, int ss, double fx, double fy, double cx, double cy,
                                const double* RC, double sphere_r, int n_rects, const double* rects,
                                double base_freq, int octaves, uint64_t seed, double background, float* out,
                                unsigned char* hit, void* stream)
{
    if (n_frames < 1 || n_frames > 65535 || W < 1 || H < 1 || ss < 1 || n_rects < 0 ||
        n_rects > SYNTH_MAX_RECTS || !RC || !out || octaves < 1)
        return 1;
    SceneParams p;
    p.fx = fx;
    p.fy = fy;
    p.cx = cx;
    p.cy = cy;
    p.sphere_r = sphere_r;
    p.base_freq = base_freq;
    p.background = background;
    p.seed = seed;
    p.W = W;
    p.H = H;
    p.ss = ss;
    p.octaves = octaves;
    p.n_rects = n_rects;
    p.F = n_frames;
    for (int i = 0; i < 11 * n_rects; ++i) p.rects[i] = rects[i];
    const dim3 grid((W + 15) / 16, (H + 15) / 16, n_frames);
    render_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(p, RC, out, hit);
    return (int)cudaGetLastError();
}
