/*
 * Seeded synthetic RGB-D scene renderer: an analytic FP64 ray caster over
 * planes and spheres with improved-Perlin fBm albedo.
 *
 * This is an INPUT GENERATOR.  It holds none of the view-synthesis method's
 * arithmetic (no difference mask, no TSDF, no splatting); both the FP64
 * oracle and the CUDA path consume what it writes.  The paper's own inputs
 * are captured multi-view video with RAFT-Stereo depth (Sec. 3, "Method");
 * these scenes stand in for them at the same image scales.
 *
 * Conventions (shared with every consumer, stated once here):
 *   camera  : world->camera x_c = R x_w + t, R row-major 3x3;
 *             pinhole K = [[fx,0,cx],[0,fy,cy],[0,0,1]], pixel (i,j) centre
 *             at integer coordinates (column i, row j); OpenCV axes.
 *   depth   : z-depth in the camera frame (metres), 0 where no surface.
 *   colour  : RGBA8, A = 255, R in the low byte of the little-endian u32.
 *
 * Noise: improved gradient noise after K. Perlin, "Improving Noise",
 * SIGGRAPH 2002 (quintic fade, 12 cube-edge gradients), with the
 * permutation drawn by a splitmix64-seeded Fisher-Yates shuffle.
 * Optional Gaussian depth noise: splitmix64 counter hash -> Box-Muller.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter-based: one 64-bit value per (seed, counter). */
static uint64_t hash_counter(uint64_t seed, uint64_t counter) {
    uint64_t s = seed ^ (counter * 0xD1B54A32D192ED03ull);
    return splitmix64(&s);
}

static double u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

typedef struct {
    int perm[512];
} noise_table;

static void noise_init(noise_table *nt, uint64_t seed) {
    int p[256];
    for (int i = 0; i < 256; ++i) p[i] = i;
    uint64_t st = seed ^ 0x5EEDF00Dull;
    for (int i = 255; i > 0; --i) {
        int j = (int)(splitmix64(&st) % (uint64_t)(i + 1));
        int tmp = p[i]; p[i] = p[j]; p[j] = tmp;
    }
    for (int i = 0; i < 512; ++i) nt->perm[i] = p[i & 255];
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }
static double lerp(double a, double b, double t) { return a + t * (b - a); }

/* Dot of the offset with one of the 12 cube-edge directions (plus 4 repeats). */
static double edge_grad(int h, double x, double y, double z) {
    switch (h & 15) {
        case 0: return x + y;   case 1: return -x + y;
        case 2: return x - y;   case 3: return -x - y;
        case 4: return x + z;   case 5: return -x + z;
        case 6: return x - z;   case 7: return -x - z;
        case 8: return y + z;   case 9: return -y + z;
        case 10: return y - z;  case 11: return -y - z;
        case 12: return x + y;  case 13: return -y + z;
        case 14: return -x + y; default: return -y - z;
    }
}

static double noise3(const noise_table *nt, double x, double y, double z) {
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int X = (int)fx & 255, Y = (int)fy & 255, Z = (int)fz & 255;
    x -= fx; y -= fy; z -= fz;
    double u = fade(x), v = fade(y), w = fade(z);
    const int *P = nt->perm;
    int A = P[X] + Y, AA = P[A] + Z, AB = P[A + 1] + Z;
    int B = P[X + 1] + Y, BA = P[B] + Z, BB = P[B + 1] + Z;
    double x0 = lerp(edge_grad(P[AA], x, y, z), edge_grad(P[BA], x - 1, y, z), u);
    double x1 = lerp(edge_grad(P[AB], x, y - 1, z), edge_grad(P[BB], x - 1, y - 1, z), u);
    double x2 = lerp(edge_grad(P[AA + 1], x, y, z - 1), edge_grad(P[BA + 1], x - 1, y, z - 1), u);
    double x3 = lerp(edge_grad(P[AB + 1], x, y - 1, z - 1), edge_grad(P[BB + 1], x - 1, y - 1, z - 1), u);
    return lerp(lerp(x0, x1, v), lerp(x2, x3, v), w);
}

static double fbm(const noise_table *nt, double x, double y, double z, double freq, int octaves) {
    double sum = 0.0, amp = 1.0, norm = 0.0;
    for (int o = 0; o < octaves; ++o) {
        sum += amp * noise3(nt, x * freq, y * freq, z * freq);
        norm += amp;
        amp *= 0.5;
        freq *= 2.0;
    }
    return sum / norm; /* roughly in [-1, 1] */
}

/* Object records: 7 doubles each.
 *   plane : nx, ny, nz, c, r, g, b   (surface n.x = c)
 *   sphere: px, py, pz, radius, r, g, b */
typedef struct {
    const double *cam;  /* fx fy cx cy R[9] t[3] */
    int W, H;
    const double *planes; int n_planes;
    const double *spheres; int n_spheres;
    const noise_table *nt;
    double tex_freq; int octaves;
    double noise_sigma; uint64_t seed; int view_id;
    uint8_t *rgba; float *depth;
    int row0, row1;
} job_t;

static void render_rows(const job_t *jb) {
    const double *c = jb->cam;
    double fx = c[0], fy = c[1], cx = c[2], cy = c[3];
    const double *R = c + 4, *t = c + 13;
    /* camera centre C = -R^T t */
    double C[3];
    for (int a = 0; a < 3; ++a) C[a] = -(R[0 * 3 + a] * t[0] + R[1 * 3 + a] * t[1] + R[2 * 3 + a] * t[2]);
    for (int j = jb->row0; j < jb->row1; ++j) {
        for (int i = 0; i < jb->W; ++i) {
            /* camera-frame direction with unit z, so the ray parameter is z-depth */
            double dc[3] = {((double)i - cx) / fx, ((double)j - cy) / fy, 1.0};
            double dw[3];
            for (int a = 0; a < 3; ++a) dw[a] = R[0 * 3 + a] * dc[0] + R[1 * 3 + a] * dc[1] + R[2 * 3 + a] * dc[2];
            double best = INFINITY;
            const double *hit_obj = NULL;
            for (int q = 0; q < jb->n_planes; ++q) {
                const double *pl = jb->planes + 7 * q;
                double nd = pl[0] * dw[0] + pl[1] * dw[1] + pl[2] * dw[2];
                if (fabs(nd) < 1e-12) continue;
                double lam = (pl[3] - (pl[0] * C[0] + pl[1] * C[1] + pl[2] * C[2])) / nd;
                if (lam > 1e-9 && lam < best) { best = lam; hit_obj = pl; }
            }
            for (int q = 0; q < jb->n_spheres; ++q) {
                const double *sp = jb->spheres + 7 * q;
                double oc[3] = {C[0] - sp[0], C[1] - sp[1], C[2] - sp[2]};
                double a2 = dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2];
                double b2 = oc[0] * dw[0] + oc[1] * dw[1] + oc[2] * dw[2];
                double c2 = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - sp[3] * sp[3];
                double disc = b2 * b2 - a2 * c2;
                if (disc < 0.0) continue;
                double sq = sqrt(disc);
                double lam = (-b2 - sq) / a2;
                if (lam <= 1e-9) lam = (-b2 + sq) / a2;
                if (lam > 1e-9 && lam < best) { best = lam; hit_obj = sp; }
            }
            size_t idx = (size_t)j * (size_t)jb->W + (size_t)i;
            uint8_t *px = jb->rgba + 4 * idx;
            if (!hit_obj) {
                px[0] = px[1] = px[2] = 0; px[3] = 255;
                jb->depth[idx] = 0.0f;
                continue;
            }
            double X[3] = {C[0] + best * dw[0], C[1] + best * dw[1], C[2] + best * dw[2]};
            /* texture lives on the surface, so for spheres use object-local coordinates:
               a moving sphere carries its texture with it */
            double tx = X[0], ty = X[1], tz = X[2];
            int is_sphere = (hit_obj >= jb->spheres && hit_obj < jb->spheres + 7 * jb->n_spheres);
            if (is_sphere) { tx -= hit_obj[0]; ty -= hit_obj[1]; tz -= hit_obj[2]; }
            double n = fbm(jb->nt, tx + 17.0, ty + 31.0, tz + 47.0, jb->tex_freq, jb->octaves);
            double shade = 0.35 + 0.65 * (0.5 + 0.5 * n);
            for (int ch = 0; ch < 3; ++ch) {
                double v = hit_obj[4 + ch] * shade;
                v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
                px[ch] = (uint8_t)lrint(255.0 * v);
            }
            px[3] = 255;
            double d = best;
            if (jb->noise_sigma > 0.0) {
                uint64_t ctr = ((uint64_t)(uint32_t)jb->view_id << 40) ^ (uint64_t)idx;
                double u1 = u01(hash_counter(jb->seed, 2 * ctr));
                double u2 = u01(hash_counter(jb->seed, 2 * ctr + 1));
                d += jb->noise_sigma * sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            }
            jb->depth[idx] = (float)d;
        }
    }
}

static void *render_thread(void *arg) { render_rows((const job_t *)arg); return NULL; }

/* Render one camera.  Returns 0 on success, -1 on bad arguments. */
int synth_render(const double *cam, int W, int H,
                 const double *planes, int n_planes,
                 const double *spheres, int n_spheres,
                 uint64_t tex_seed, double tex_freq, int octaves,
                 uint64_t noise_seed, double noise_sigma, int view_id,
                 int n_threads, uint8_t *rgba_out, float *depth_out) {
    if (!cam || W <= 0 || H <= 0 || !rgba_out || !depth_out) return -1;
    noise_table nt;
    noise_init(&nt, tex_seed);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads > H) n_threads = H;
    job_t jobs[256];
    pthread_t th[256];
    for (int k = 0; k < n_threads; ++k) {
        job_t jb = {cam, W, H, planes, n_planes, spheres, n_spheres, &nt, tex_freq, octaves,
                    noise_sigma, noise_seed, view_id, rgba_out, depth_out,
                    (int)((long)H * k / n_threads), (int)((long)H * (k + 1) / n_threads)};
        jobs[k] = jb;
    }
    int started = 0;
    for (int k = 1; k < n_threads; ++k) {
        if (pthread_create(&th[k], NULL, render_thread, &jobs[k]) != 0) break;
        started = k;
    }
    render_rows(&jobs[0]);
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    for (int k = started + 1; k < n_threads; ++k) render_rows(&jobs[k]);
    return 0;
}
