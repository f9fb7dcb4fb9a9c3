/* FP64 CPU oracle for the neural six-way lightmap hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Plain, slow,
 * direct loops; no blocking or fusion.  Each function cites the passage of the
 * paper it follows.
 *
 * Precision.  All radiometric arithmetic is binary64.  The ray geometry that
 * decides integers (the number of view samples N, the number of shadow samples
 * K, the sample positions) is evaluated in binary32 with one rounding per
 * operation in a fixed order, because the GPU kernel takes those decisions in
 * binary32; both sides must take an integer decision in the same precision.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Parity pins (tests): empty volume; constant cube closed form (front, top,
 * bottom geometric sums, T = exp(-sigma L)); linear density field (trilinear is
 * exact, optical depth is an arithmetic series); vertical flip symmetry;
 * mask-all = empty; Henyey-Greenstein normalisation; convolution, transposed
 * convolution, pooling and LayerNorm against PyTorch float64; NAFBlock with
 * beta = gamma = 0 is the identity; shading selects one plane on axis lights
 * and is linear; the fine-step reference against the slab closed form.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* binary32 camera geometry (Sec. 4.2: view rays along -omega from x)        */
/* ------------------------------------------------------------------------- */

typedef struct {
  float eye[3], r[3], u[3], f[3];
  float ax, ay;           /* screen extents: ortho (height*W/H, height), persp 2tan(fov/2)*(W/H, 1) */
  int kind, W, H;
} cam_frame;

/* Camera basis in binary64, rounded once to binary32: f = normalize(target -
 * eye), r = normalize(f x up), u = r x f (right-handed, Y up world). */
static void cam_setup(const nslo_camera* c, cam_frame* fr) {
  double fx = (double)c->target[0] - (double)c->eye[0];
  double fy = (double)c->target[1] - (double)c->eye[1];
  double fz = (double)c->target[2] - (double)c->eye[2];
  double fl = sqrt(fx * fx + fy * fy + fz * fz);
  fx /= fl; fy /= fl; fz /= fl;
  double ux = c->up[0], uy = c->up[1], uz = c->up[2];
  double rx = fy * uz - fz * uy, ry = fz * ux - fx * uz, rz = fx * uy - fy * ux;
  double rl = sqrt(rx * rx + ry * ry + rz * rz);
  rx /= rl; ry /= rl; rz /= rl;
  double vx = ry * fz - rz * fy, vy = rz * fx - rx * fz, vz = rx * fy - ry * fx;
  for (int k = 0; k < 3; ++k) fr->eye[k] = c->eye[k];
  fr->f[0] = (float)fx; fr->f[1] = (float)fy; fr->f[2] = (float)fz;
  fr->r[0] = (float)rx; fr->r[1] = (float)ry; fr->r[2] = (float)rz;
  fr->u[0] = (float)vx; fr->u[1] = (float)vy; fr->u[2] = (float)vz;
  fr->kind = c->kind; fr->W = c->width; fr->H = c->height;
  if (c->kind == 0) {
    fr->ax = (float)(((double)c->ortho_height * (double)c->width) / (double)c->height);
    fr->ay = c->ortho_height;
  } else {
    double k = 2.0 * tan(((double)c->fov_y_deg * PI_D / 180.0) * 0.5);
    fr->ax = (float)((k * (double)c->width) / (double)c->height);
    fr->ay = (float)k;
  }
}

/* Pixel (i, j) -> ray origin o and unit direction d (binary32). */
static void pixel_ray(const cam_frame* fr, int i, int j, float o[3], float d[3]) {
  float sx = ((float)i + 0.5f) / (float)fr->W - 0.5f;
  float sy = 0.5f - ((float)j + 0.5f) / (float)fr->H;
  float a = sx * fr->ax;
  float b = sy * fr->ay;
  if (fr->kind == 0) {
    for (int k = 0; k < 3; ++k) {
      float t1 = a * fr->r[k];
      float t2 = b * fr->u[k];
      o[k] = (fr->eye[k] + t1) + t2;
      d[k] = fr->f[k];
    }
  } else {
    float v[3];
    for (int k = 0; k < 3; ++k) {
      float t1 = a * fr->r[k];
      float t2 = b * fr->u[k];
      v[k] = (fr->f[k] + t1) + t2;
      o[k] = fr->eye[k];
    }
    float s0 = v[0] * v[0];
    float s1 = v[1] * v[1];
    float s2 = v[2] * v[2];
    float len = sqrtf((s0 + s1) + s2);
    for (int k = 0; k < 3; ++k) d[k] = v[k] / len;
  }
}

/* Slab clip of the ray against the closed box [0,n]; returns 0 on a miss. */
static int clip_box(const float o[3], const float d[3], const float n[3], float* tin,
                    float* tout) {
  float tn = -INFINITY, tf = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.0f) {
      float ta = (0.0f - o[k]) / d[k];
      float tb = (n[k] - o[k]) / d[k];
      float lo = ta < tb ? ta : tb;
      float hi = ta < tb ? tb : ta;
      if (lo > tn) tn = lo;
      if (hi < tf) tf = hi;
    } else if (o[k] < 0.0f || o[k] > n[k]) {
      return 0;
    }
  }
  if (tn < 0.0f) tn = 0.0f;
  if (!(tf > tn)) return 0;
  *tin = tn;
  *tout = tf;
  return 1;
}

/* Distance from p to the exit of the closed box along unit direction s. */
static float exit_distance(const float p[3], const float s[3], const float n[3]) {
  float te = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (s[k] > 0.0f) {
      float t = (n[k] - p[k]) / s[k];
      if (t < te) te = t;
    } else if (s[k] < 0.0f) {
      float t = (0.0f - p[k]) / s[k];
      if (t < te) te = t;
    }
  }
  return te;
}

/* 32-bit PCG hash, from Jarzynski & Olano, "Hash Functions for GPU Rendering",
 * JCGT 9(3), 2020: an LCG step followed by a random xorshift and a multiply. */
uint32_t nslo_pcg_hash(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

/* Jitter u in [0,1) for pixel (i,j): top 24 bits of a hash chain. */
static float pixel_jitter(const nslo_march_opts* op, int i, int j, int W) {
  if (!op->jitter) return 0.0f;
  uint32_t key = nslo_pcg_hash(op->frame + nslo_pcg_hash(op->seed));
  uint32_t hv = nslo_pcg_hash((uint32_t)(j * W + i) + key);
  return (float)(hv >> 8) * (1.0f / 16777216.0f);
}

/* ------------------------------------------------------------------------- */
/* density field (Sec. 4.2: sigma_s stored in a 3D texture)                   */
/* ------------------------------------------------------------------------- */

typedef struct {
  const float* rho;
  const uint8_t* mask;
  int nx, ny, nz;
  double scale;
  float n[3];
} field;

static double voxel(const field* F, int i, int j, int k) {
  size_t idx = ((size_t)k * F->ny + j) * F->nx + i;
  if (F->mask && F->mask[idx]) return 0.0;
  return F->scale * (double)F->rho[idx];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* sigma(p): 0 outside the closed box; trilinear interpolation of the masked,
 * scaled voxels at q = p - 0.5 with clamp-to-edge indices inside it. */
static double sigma_at(const field* F, const float p[3]) {
  for (int k = 0; k < 3; ++k)
    if (!(p[k] >= 0.0f && p[k] <= F->n[k])) return 0.0;
  double q[3] = {(double)p[0] - 0.5, (double)p[1] - 0.5, (double)p[2] - 0.5};
  int i0[3];
  double t[3];
  for (int k = 0; k < 3; ++k) {
    double fl = floor(q[k]);
    i0[k] = (int)fl;
    t[k] = q[k] - fl;
  }
  int lim[3] = {F->nx - 1, F->ny - 1, F->nz - 1};
  int ia[3], ib[3];
  for (int k = 0; k < 3; ++k) {
    ia[k] = clampi(i0[k], 0, lim[k]);
    ib[k] = clampi(i0[k] + 1, 0, lim[k]);
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
        acc += w * voxel(F, dx ? ib[0] : ia[0], dy ? ib[1] : ia[1], dz ? ib[2] : ia[2]);
      }
  return acc;
}

double nslo_sample_sigma(const float* density, const uint8_t* mask, int nx, int ny, int nz,
                         double sigma_scale, const float p[3]) {
  field F = {density, mask, nx, ny, nz, sigma_scale, {(float)nx, (float)ny, (float)nz}};
  return sigma_at(&F, p);
}

/* Henyey-Greenstein phase function; cos_theta is the cosine between the light's
 * propagation direction and the scattered direction (toward the camera). */
double nslo_hg_phase(double g, double cos_theta) {
  double den = 1.0 + g * g - 2.0 * g * cos_theta;
  return (1.0 - g * g) / (4.0 * PI_D * den * sqrt(den));
}

/* ------------------------------------------------------------------------- */
/* Guiding map: Alg. 1 with the surrogate lights of Eq. approx                */
/* ------------------------------------------------------------------------- */

/* Transmittance from p toward direction s (front/top/bottom light) by a march
 * at step h to the box exit: T = exp(-h sum_k sigma(p + k h s)).  Stops once
 * the running transmittance is below t_min (checked after each step). */
static double shadow_T(const field* F, const float p[3], const float s[3], float h,
                       double t_min, double margin, int64_t* nsamp, int* near_flag) {
  float te = exit_distance(p, s, F->n);
  int K = 0;
  if (te > 0.0f) {
    float kf = floorf(te / h);
    K = (int)kf;
  }
  double tau = 0.0, T = 1.0;
  for (int k = 1; k <= K; ++k) {
    float kh = (float)k * h;
    float q[3];
    for (int c = 0; c < 3; ++c) {
      float st = kh * s[c];
      q[c] = p[c] + st;
    }
    tau += sigma_at(F, q) * (double)h;
    ++*nsamp;
    T = exp(-tau);
    if (t_min > 0.0) {
      if (fabs(T - t_min) <= margin * t_min) *near_flag = 1;
      if (T < t_min) break;
    }
  }
  return T;
}

/* Trilinear value of a cell-centred volume v [nz][ny][nx] at p (inside the
 * box): q = p - 0.5 with clamp-to-edge indices, as for the density. */
static double vol_at(const double* v, int nx, int ny, int nz, const float p[3]) {
  double q[3] = {(double)p[0] - 0.5, (double)p[1] - 0.5, (double)p[2] - 0.5};
  int i0[3];
  double t[3];
  for (int k = 0; k < 3; ++k) {
    double fl = floor(q[k]);
    i0[k] = (int)fl;
    t[k] = q[k] - fl;
  }
  int lim[3] = {nx - 1, ny - 1, nz - 1};
  int ia[3], ib[3];
  for (int k = 0; k < 3; ++k) {
    ia[k] = clampi(i0[k], 0, lim[k]);
    ib[k] = clampi(i0[k] + 1, 0, lim[k]);
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
        size_t idx = ((size_t)(dz ? ib[2] : ia[2]) * ny + (dy ? ib[1] : ia[1])) * nx + (dx ? ib[0] : ia[0]);
        acc += w * v[idx];
      }
  return acc;
}

int nslo_guide(const float* density, const uint8_t* mask, int nx, int ny, int nz,
               double sigma_scale, const nslo_camera* cam, float h,
               const nslo_march_opts* op, double* guide, int64_t* samples, uint8_t* flags) {
  if (!cam) return 1;
  return nslo_guide_rows(density, mask, nx, ny, nz, sigma_scale, cam, h, op, 0, cam->height,
                         guide, samples, flags);
}

int nslo_guide_rows(const float* density, const uint8_t* mask, int nx, int ny, int nz,
                    double sigma_scale, const nslo_camera* cam, float h,
                    const nslo_march_opts* op, int row0, int row1, double* guide,
                    int64_t* samples, uint8_t* flags) {
  if (!density || !cam || !op || !guide || nx <= 0 || ny <= 0 || nz <= 0 || !(h > 0.0f))
    return 1;
  if (row0 < 0 || row1 > cam->height || row0 > row1) return 1;
  field F = {density, mask, nx, ny, nz, sigma_scale, {(float)nx, (float)ny, (float)nz}};
  cam_frame fr;
  cam_setup(cam, &fr);
  const int W = cam->width, H = cam->height;
  const size_t plane = (size_t)W * H;
  const double t_min = op->t_min, margin = op->margin;
  const double g = op->phase_g;

  /* shadow_volume: the top/bottom (or right/left) transmittances marched once
   * from every voxel centre, as from a view sample */
  double* volT = NULL;
  double* volB = NULL;
  if (op->shadow_volume && op->light_set != 1) {
    const size_t nv = (size_t)nx * ny * nz;
    volT = (double*)malloc(nv * sizeof(double));
    volB = (double*)malloc(nv * sizeof(double));
    if (!volT || !volB) { free(volT); free(volB); return 1; }
    const float* sd = op->light_set == 2 ? fr.r : fr.u;
    const float st[3] = {sd[0], sd[1], sd[2]}, sb[3] = {-sd[0], -sd[1], -sd[2]};
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
          int64_t ns_unused = 0;
          int nf_unused = 0;
          const size_t idx = ((size_t)k * ny + j) * nx + i;
          volT[idx] = shadow_T(&F, p, st, h, t_min, margin, &ns_unused, &nf_unused);
          volB[idx] = shadow_T(&F, p, sb, h, t_min, margin, &ns_unused, &nf_unused);
        }
  }

#pragma omp parallel for schedule(dynamic, 4)
  for (int j = row0; j < row1; ++j) {
    for (int i = 0; i < W; ++i) {
      size_t pix = (size_t)j * W + i;
      float o[3], d[3], tin, tout;
      pixel_ray(&fr, i, j, o, d);
      double L = 0.0, T = 1.0, D = 0.0;
      int64_t ns = 0;
      int near_term = 0, near_depth = 0;
      if (clip_box(o, d, F.n, &tin, &tout)) {
        float u = pixel_jitter(op, i, j, W);
        float span = (tout - tin) / h;
        int N = (int)floorf(span + u);
        /* surrogate lights (Eq. approx): front = toward the camera (-d), top =
         * camera up (+u), bottom = -u; HG cosines against the view ray.  The
         * ablation sets of Sec. 5 replace the side pair by right (+r) / left
         * (-r), or drop it (front only). */
        const int side_on = op->light_set != 1;
        const float* sd = op->light_set == 2 ? fr.r : fr.u;
        float s_top[3] = {sd[0], sd[1], sd[2]};
        float s_bot[3] = {-sd[0], -sd[1], -sd[2]};
        double cu = (double)d[0] * sd[0] + (double)d[1] * sd[1] + (double)d[2] * sd[2];
        double P_f = nslo_hg_phase(g, -1.0);
        double P_t = nslo_hg_phase(g, cu);
        double P_b = nslo_hg_phase(g, -cu);
        double tau = 0.0;
        for (int n = 1; n <= N; ++n) {
          float tn_off = ((float)n - u) * h;
          float tn = tin + tn_off;
          float p[3];
          for (int c = 0; c < 3; ++c) {
            float st = tn * d[c];
            p[c] = o[c] + st;
          }
          double sg = sigma_at(&F, p);
          ++ns;
          if (D == 0.0) {
            if (fabs(sg - (double)op->tau_depth) <= margin * (double)op->tau_depth) near_depth = 1;
            if (sg > (double)op->tau_depth) D = (double)n * (double)h;
          }
          double A = op->segment_exact ? T * (1.0 - exp(-sg * (double)h)) : T * sg * (double)h;
          /* sigma_n = 0 gives A_n = 0, so A_n L_n vanishes whatever L_n is: the
           * shadow rays of such a sample are not marched (and not counted) */
          double Tt = 1.0, Tb = 1.0;
          if (sg > 0.0 && side_on) {
            if (volT) {
              Tt = vol_at(volT, nx, ny, nz, p);
              Tb = vol_at(volB, nx, ny, nz, p);
            } else {
              Tt = shadow_T(&F, p, s_top, h, t_min, margin, &ns, &near_term);
              Tb = shadow_T(&F, p, s_bot, h, t_min, margin, &ns, &near_term);
            }
          }
          double Ln = P_f * op->surrogate_I[0] * T;
          if (side_on) Ln += P_t * op->surrogate_I[1] * Tt + P_b * op->surrogate_I[2] * Tb;
          L += A * Ln;
          tau += sg * (double)h;
          T = exp(-tau);
          if (t_min > 0.0) {
            if (fabs(T - t_min) <= margin * t_min) near_term = 1;
            if (T < t_min) break;
          }
        }
      }
      guide[pix] = L;
      guide[plane + pix] = T;
      guide[2 * plane + pix] = D;
      if (samples) samples[pix] = ns;
      if (flags) flags[pix] = (uint8_t)(near_term | (near_depth << 1));
    }
  }
  free(volT);
  free(volB);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Fine-step six-light reference (single scattering, Sec. 3 Eq. RE/scatter)   */
/* ------------------------------------------------------------------------- */

/* Optical depth from p toward s to the box exit, midpoint rule with segments
 * of length at most hf. */
static double light_tau(const field* F, const float p[3], const double s[3], double hf) {
  double pd[3] = {p[0], p[1], p[2]};
  double te = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (s[k] > 0.0) te = fmin(te, ((double)F->n[k] - pd[k]) / s[k]);
    else if (s[k] < 0.0) te = fmin(te, (0.0 - pd[k]) / s[k]);
  }
  if (!(te > 0.0)) return 0.0;
  int M = (int)ceil(te / hf);
  double hs = te / M, tau = 0.0;
  for (int m = 1; m <= M; ++m) {
    double t = ((double)m - 0.5) * hs;
    float q[3] = {(float)(pd[0] + t * s[0]), (float)(pd[1] + t * s[1]), (float)(pd[2] + t * s[2])};
    tau += sigma_at(F, q) * hs;
  }
  return tau;
}

int nslo_reference_lightmaps(const float* density, const uint8_t* mask, int nx, int ny, int nz,
                             double sigma_scale, const nslo_camera* cam, double hf,
                             double g, double* out) {
  return nslo_reference_lightmaps_rows(density, mask, nx, ny, nz, sigma_scale, cam, hf, g, 0,
                                       cam ? cam->height : 0, out);
}

int nslo_reference_lightmaps_rows(const float* density, const uint8_t* mask, int nx, int ny, int nz,
                                  double sigma_scale, const nslo_camera* cam, double hf, double g,
                                  int row0, int row1, double* out) {
  if (!density || !cam || !out || !(hf > 0.0)) return 1;
  if (row0 < 0 || row1 > cam->height || row0 > row1) return 1;
  field F = {density, mask, nx, ny, nz, sigma_scale, {(float)nx, (float)ny, (float)nz}};
  cam_frame fr;
  cam_setup(cam, &fr);
  const int W = cam->width, H = cam->height;
  const size_t plane = (size_t)W * H;
  (void)H;
  /* toward-light directions in the camera frame: +X right, -X, +Y up, -Y,
   * +Z back (behind the smoke, along the view direction), -Z front */
  double dirs[6][3];
  for (int k = 0; k < 3; ++k) {
    dirs[0][k] = fr.r[k]; dirs[1][k] = -(double)fr.r[k];
    dirs[2][k] = fr.u[k]; dirs[3][k] = -(double)fr.u[k];
    dirs[4][k] = fr.f[k]; dirs[5][k] = -(double)fr.f[k];
  }
#pragma omp parallel for schedule(dynamic, 2)
  for (int j = row0; j < row1; ++j) {
    for (int i = 0; i < W; ++i) {
      size_t pix = (size_t)j * W + i;
      float o[3], d[3], tin, tout;
      pixel_ray(&fr, i, j, o, d);
      double Lp[6] = {0, 0, 0, 0, 0, 0}, T = 1.0;
      if (clip_box(o, d, F.n, &tin, &tout)) {
        double chord = (double)tout - (double)tin;
        int M = (int)ceil(chord / hf);
        double hs = chord / M, tau = 0.0;
        for (int m = 1; m <= M; ++m) {
          double t = (double)tin + ((double)m - 0.5) * hs;
          float p[3] = {(float)((double)o[0] + t * d[0]), (float)((double)o[1] + t * d[1]),
                        (float)((double)o[2] + t * d[2])};
          double sg = sigma_at(&F, p);
          if (sg > 0.0) {
            double w = T * (1.0 - exp(-sg * hs));
            for (int l = 0; l < 6; ++l) {
              double cth = dirs[l][0] * d[0] + dirs[l][1] * d[1] + dirs[l][2] * d[2];
              Lp[l] += w * nslo_hg_phase(g, cth) * exp(-light_tau(&F, p, dirs[l], hf));
            }
          }
          tau += sg * hs;
          T = exp(-tau);
        }
      }
      for (int l = 0; l < 6; ++l) out[l * plane + pix] = Lp[l];
      out[6 * plane + pix] = T;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Network (Sec. 4.3): UNet encoder/decoder + four NAFBlock channel adapters  */
/* ------------------------------------------------------------------------- */

/* 'same' convolution, zero padding (k-1)/2, w [cout][cin][k][k], planar NCHW. */
void nslo_conv2d(const double* in, int cin, int H, int W, const double* w, const double* b,
                 int cout, int k, double* out) {
  int pad = (k - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int co = 0; co < cout; ++co) {
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double acc = b ? b[co] : 0.0;
        for (int ci = 0; ci < cin; ++ci)
          for (int ky = 0; ky < k; ++ky) {
            int yy = y + ky - pad;
            if (yy < 0 || yy >= H) continue;
            for (int kx = 0; kx < k; ++kx) {
              int xx = x + kx - pad;
              if (xx < 0 || xx >= W) continue;
              acc += w[((size_t)(co * cin + ci) * k + ky) * k + kx] *
                     in[((size_t)ci * H + yy) * W + xx];
            }
          }
        out[((size_t)co * H + y) * W + x] = acc;
      }
  }
}

/* 2x2 stride-2 transposed convolution, w [cin][cout][2][2]: output pixel
 * (2y+a, 2x+b) = bias + sum_ci w[ci][co][a][b] in[ci][y][x]. */
void nslo_conv_transpose2x2(const double* in, int cin, int H, int W, const double* w,
                            const double* b, int cout, double* out) {
  int H2 = 2 * H, W2 = 2 * W;
#pragma omp parallel for schedule(static)
  for (int co = 0; co < cout; ++co)
    for (int y = 0; y < H2; ++y)
      for (int x = 0; x < W2; ++x) {
        int a = y & 1, bb = x & 1;
        double acc = b ? b[co] : 0.0;
        for (int ci = 0; ci < cin; ++ci)
          acc += w[((size_t)(ci * cout + co) * 2 + a) * 2 + bb] *
                 in[((size_t)ci * H + y / 2) * W + x / 2];
        out[((size_t)co * H2 + y) * W2 + x] = acc;
      }
}

void nslo_maxpool2(const double* in, int C, int H, int W, double* out) {
  int H2 = H / 2, W2 = W / 2;
  for (int c = 0; c < C; ++c)
    for (int y = 0; y < H2; ++y)
      for (int x = 0; x < W2; ++x) {
        const double* p = in + ((size_t)c * H + 2 * y) * W + 2 * x;
        double m = p[0];
        if (p[1] > m) m = p[1];
        if (p[W] > m) m = p[W];
        if (p[W + 1] > m) m = p[W + 1];
        out[((size_t)c * H2 + y) * W2 + x] = m;
      }
}

/* LayerNorm over channels at every pixel (NAFNet's LayerNorm2d): biased
 * variance, eps inside the square root, then per-channel affine. */
void nslo_layernorm(const double* in, int C, int H, int W, const double* g, const double* b,
                    double eps, double* out) {
  size_t plane = (size_t)H * W;
  for (size_t p = 0; p < plane; ++p) {
    double mu = 0.0;
    for (int c = 0; c < C; ++c) mu += in[c * plane + p];
    mu /= C;
    double var = 0.0;
    for (int c = 0; c < C; ++c) {
      double dv = in[c * plane + p] - mu;
      var += dv * dv;
    }
    var /= C;
    double inv = 1.0 / sqrt(var + eps);
    for (int c = 0; c < C; ++c) out[c * plane + p] = (in[c * plane + p] - mu) * inv * g[c] + b[c];
  }
}

/* depthwise 3x3 'same' convolution, w [C][1][3][3] */
void nslo_dwconv3(const double* in, int C, int H, int W, const double* w, const double* b,
                  double* out) {
  for (int c = 0; c < C; ++c)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double acc = b[c];
        for (int ky = 0; ky < 3; ++ky) {
          int yy = y + ky - 1;
          if (yy < 0 || yy >= H) continue;
          for (int kx = 0; kx < 3; ++kx) {
            int xx = x + kx - 1;
            if (xx < 0 || xx >= W) continue;
            acc += w[c * 9 + ky * 3 + kx] * in[((size_t)c * H + yy) * W + xx];
          }
        }
        out[((size_t)c * H + y) * W + x] = acc;
      }
}

/* simple gate: first half of the channels times the second half */
static void simple_gate(const double* in, int C2, size_t plane, double* out) {
  int C = C2 / 2;
  for (int c = 0; c < C; ++c)
    for (size_t p = 0; p < plane; ++p) out[c * plane + p] = in[c * plane + p] * in[(c + C) * plane + p];
}

int64_t nslo_nafblock_params(int C) {
  /* ln1 (2C), pw1 (2C*C + 2C), dw (2C*9 + 2C), sca (C*C + C), pw2 (C*C + C),
   * beta (C), ln2 (2C), ffn1 (2C*C + 2C), ffn2 (C*C + C), gamma (C) */
  return (int64_t)2 * C + (2 * C * C + 2 * C) + (18 * C + 2 * C) + (C * C + C) + (C * C + C) + C +
         2 * C + (2 * C * C + 2 * C) + (C * C + C) + C;
}

/* NAFBlock (Chen et al. 2022, the adapter block named in Sec. 4.3):
 *   y = x + beta  * pw2(SCA(SG(dw3x3(pw1(LN1(x))))))
 *   z = y + gamma * ffn2(SG(ffn1(LN2(y))))
 * SG(a|b) = a*b over the two channel halves; SCA(v) = v * (W_sca mean_HW(v) + b). */
int nslo_nafblock(const double* in, int C, int H, int W, const double* P, double* out) {
  size_t plane = (size_t)H * W;
  const double *ln1w = P, *ln1b = P + C;
  P += 2 * C;
  const double *pw1w = P, *pw1b = P + 2 * C * C;
  P += 2 * C * C + 2 * C;
  const double *dww = P, *dwb = P + 18 * C;
  P += 20 * C;
  const double *scaw = P, *scab = P + C * C;
  P += C * C + C;
  const double *pw2w = P, *pw2b = P + C * C;
  P += C * C + C;
  const double* beta = P;
  P += C;
  const double *ln2w = P, *ln2b = P + C;
  P += 2 * C;
  const double *f1w = P, *f1b = P + 2 * C * C;
  P += 2 * C * C + 2 * C;
  const double *f2w = P, *f2b = P + C * C;
  P += C * C + C;
  const double* gamma = P;

  double* t_ln = malloc(sizeof(double) * C * plane);
  double* t_2c = malloc(sizeof(double) * 2 * C * plane);
  double* t_2c_b = malloc(sizeof(double) * 2 * C * plane);
  double* t_c = malloc(sizeof(double) * C * plane);
  double* t_c2 = malloc(sizeof(double) * C * plane);
  double* y = malloc(sizeof(double) * C * plane);
  if (!t_ln || !t_2c || !t_2c_b || !t_c || !t_c2 || !y) return 2;

  nslo_layernorm(in, C, H, W, ln1w, ln1b, 1e-6, t_ln);
  nslo_conv2d(t_ln, C, H, W, pw1w, pw1b, 2 * C, 1, t_2c);
  nslo_dwconv3(t_2c, 2 * C, H, W, dww, dwb, t_2c_b);
  simple_gate(t_2c_b, 2 * C, plane, t_c);
  /* simplified channel attention */
  double* mean = malloc(sizeof(double) * C);
  double* att = malloc(sizeof(double) * C);
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (size_t p = 0; p < plane; ++p) s += t_c[c * plane + p];
    mean[c] = s / (double)plane;
  }
  for (int co = 0; co < C; ++co) {
    double s = scab[co];
    for (int ci = 0; ci < C; ++ci) s += scaw[co * C + ci] * mean[ci];
    att[co] = s;
  }
  for (int c = 0; c < C; ++c)
    for (size_t p = 0; p < plane; ++p) t_c[c * plane + p] *= att[c];
  nslo_conv2d(t_c, C, H, W, pw2w, pw2b, C, 1, t_c2);
  for (int c = 0; c < C; ++c)
    for (size_t p = 0; p < plane; ++p) y[c * plane + p] = in[c * plane + p] + beta[c] * t_c2[c * plane + p];
  /* feed-forward half */
  nslo_layernorm(y, C, H, W, ln2w, ln2b, 1e-6, t_ln);
  nslo_conv2d(t_ln, C, H, W, f1w, f1b, 2 * C, 1, t_2c);
  simple_gate(t_2c, 2 * C, plane, t_c);
  nslo_conv2d(t_c, C, H, W, f2w, f2b, C, 1, t_c2);
  for (int c = 0; c < C; ++c)
    for (size_t p = 0; p < plane; ++p) out[c * plane + p] = y[c * plane + p] + gamma[c] * t_c2[c * plane + p];
  free(mean); free(att);
  free(t_ln); free(t_2c); free(t_2c_b); free(t_c); free(t_c2); free(y);
  return 0;
}

static void relu_inplace(double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (v[i] < 0.0) v[i] = 0.0;
}

typedef struct { const double* p; int64_t left; } cursor;

static const double* take(cursor* c, int64_t n) {
  if (c->left < n) return NULL;
  const double* r = c->p;
  c->p += n;
  c->left -= n;
  return r;
}

/* conv3x3 + ReLU with parameters from the cursor */
static int conv3_relu(cursor* cur, const double* in, int cin, int H, int W, int cout, double* out) {
  const double* w = take(cur, (int64_t)cout * cin * 9);
  const double* b = take(cur, cout);
  if (!w || !b) return 3;
  nslo_conv2d(in, cin, H, W, w, b, cout, 3, out);
  relu_inplace(out, (size_t)cout * H * W);
  return 0;
}

/* The four channel adapters (F&B, L&R, U&D, A&E in that order), each a
 * NAFBlock on F followed by a 1x1 conv to two output planes. */
static int adapters_forward(cursor* cur, const double* F, int c1, int H, int W, double* z,
                            double* out) {
  static const int plane_of[4][2] = {{4, 5}, {0, 1}, {2, 3}, {6, 7}};
  const size_t P0 = (size_t)H * W;
  int64_t nb = nslo_nafblock_params(c1);
  for (int a = 0; a < 4; ++a) {
    const double* bp = take(cur, nb);
    const double* hw = take(cur, 2 * c1);
    const double* hb = take(cur, 2);
    if (!bp || !hw || !hb) return 3;
    int rc = nslo_nafblock(F, c1, H, W, bp, z);
    if (rc) return rc;
    for (int oc = 0; oc < 2; ++oc) {
      double* dst = out + (size_t)plane_of[a][oc] * P0;
      for (size_t p = 0; p < P0; ++p) {
        double s = hb[oc];
        for (int ci = 0; ci < c1; ++ci) s += hw[oc * c1 + ci] * z[ci * P0 + p];
        dst[p] = s;
      }
    }
  }
  return 0;
}

/* The lightmap generator of Sec. 4.3 / Fig. 3: a four-level UNet (widths
 * c0*{1,2,4,8}, two 3x3 conv+ReLU per level, 2x2 max-pool down, 2x2 stride-2
 * transposed conv up, skip concatenated after the upsampled tensor) gives the
 * shared feature F; four NAFBlock adapters (F&B, L&R, U&D, A&E) each end in a
 * 1x1 conv to 2 channels.  Output planes [+X,-X,+Y,-Y,+Z,-Z,T,E]:
 * L&R -> 0,1; U&D -> 2,3; F&B -> 4 (+Z back), 5 (-Z front); A&E -> 6,7.
 * Input: the guide with its depth channel multiplied by depth_scale. */
int nslo_net_forward(const double* guide, int H, int W, const double* params, int64_t n_params,
                     int c0, double depth_scale, double* out) {
  if (H % 8 || W % 8 || H <= 0 || W <= 0) return 1;
  cursor cur = {params, n_params};
  const int c1 = c0, c2 = 2 * c0, c3 = 4 * c0, c4 = 8 * c0;
  size_t P0 = (size_t)H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  double* x0 = malloc(sizeof(double) * 3 * P0);
  double* a0 = malloc(sizeof(double) * c1 * P0);
  double* s1 = malloc(sizeof(double) * c1 * P0);
  double* p1 = malloc(sizeof(double) * c1 * P1);
  double* a1 = malloc(sizeof(double) * c2 * P1);
  double* s2 = malloc(sizeof(double) * c2 * P1);
  double* p2 = malloc(sizeof(double) * c2 * P2);
  double* a2 = malloc(sizeof(double) * c3 * P2);
  double* s3 = malloc(sizeof(double) * c3 * P2);
  double* p3 = malloc(sizeof(double) * c3 * P3);
  double* a3 = malloc(sizeof(double) * c4 * P3);
  double* bt = malloc(sizeof(double) * c4 * P3);
  double* cat = malloc(sizeof(double) * 2 * c1 * P0 + sizeof(double) * c4 * P2);
  double* d = malloc(sizeof(double) * c1 * P0 * 2 + sizeof(double) * c4 * P2);
  double* F = malloc(sizeof(double) * c1 * P0);
  double* z = malloc(sizeof(double) * c1 * P0);
  int rc = 0;
  if (!x0 || !a0 || !s1 || !p1 || !a1 || !s2 || !p2 || !a2 || !s3 || !p3 || !a3 || !bt || !cat ||
      !d || !F || !z) { rc = 2; goto done; }

  memcpy(x0, guide, sizeof(double) * 2 * P0);
  for (size_t p = 0; p < P0; ++p) x0[2 * P0 + p] = guide[2 * P0 + p] * depth_scale;

  /* encoder */
  if ((rc = conv3_relu(&cur, x0, 3, H, W, c1, a0))) goto done;
  if ((rc = conv3_relu(&cur, a0, c1, H, W, c1, s1))) goto done;
  nslo_maxpool2(s1, c1, H, W, p1);
  if ((rc = conv3_relu(&cur, p1, c1, H1, W1, c2, a1))) goto done;
  if ((rc = conv3_relu(&cur, a1, c2, H1, W1, c2, s2))) goto done;
  nslo_maxpool2(s2, c2, H1, W1, p2);
  if ((rc = conv3_relu(&cur, p2, c2, H2, W2, c3, a2))) goto done;
  if ((rc = conv3_relu(&cur, a2, c3, H2, W2, c3, s3))) goto done;
  nslo_maxpool2(s3, c3, H2, W2, p3);
  if ((rc = conv3_relu(&cur, p3, c3, H3, W3, c4, a3))) goto done;
  if ((rc = conv3_relu(&cur, a3, c4, H3, W3, c4, bt))) goto done;

  /* decoder: level 3 */
  {
    const double* w = take(&cur, (int64_t)c4 * c3 * 4);
    const double* b = take(&cur, c3);
    if (!w || !b) { rc = 3; goto done; }
    nslo_conv_transpose2x2(bt, c4, H3, W3, w, b, c3, cat);           /* upsampled first */
    memcpy(cat + (size_t)c3 * P2, s3, sizeof(double) * c3 * P2);     /* skip second */
    if ((rc = conv3_relu(&cur, cat, 2 * c3, H2, W2, c3, d))) goto done;
    if ((rc = conv3_relu(&cur, d, c3, H2, W2, c3, a2))) goto done;
  }
  /* level 2 */
  {
    const double* w = take(&cur, (int64_t)c3 * c2 * 4);
    const double* b = take(&cur, c2);
    if (!w || !b) { rc = 3; goto done; }
    nslo_conv_transpose2x2(a2, c3, H2, W2, w, b, c2, cat);
    memcpy(cat + (size_t)c2 * P1, s2, sizeof(double) * c2 * P1);
    if ((rc = conv3_relu(&cur, cat, 2 * c2, H1, W1, c2, d))) goto done;
    if ((rc = conv3_relu(&cur, d, c2, H1, W1, c2, a1))) goto done;
  }
  /* level 1 */
  {
    const double* w = take(&cur, (int64_t)c2 * c1 * 4);
    const double* b = take(&cur, c1);
    if (!w || !b) { rc = 3; goto done; }
    nslo_conv_transpose2x2(a1, c2, H1, W1, w, b, c1, cat);
    memcpy(cat + (size_t)c1 * P0, s1, sizeof(double) * c1 * P0);
    if ((rc = conv3_relu(&cur, cat, 2 * c1, H, W, c1, d))) goto done;
    if ((rc = conv3_relu(&cur, d, c1, H, W, c1, F))) goto done;
  }
  /* channel adapters */
  if ((rc = adapters_forward(&cur, F, c1, H, W, z, out))) goto done;
  if (cur.left != 0) rc = 4;
done:
  free(x0); free(a0); free(s1); free(p1); free(a1); free(s2); free(p2); free(a2); free(s3);
  free(p3); free(a3); free(bt); free(cat); free(d); free(F); free(z);
  return rc;
}


/* ------------------------------------------------------------------------- */
/* FP8 E4M3 network (precision form; no counterpart in the paper)            */
/* ------------------------------------------------------------------------- */

/* IEEE binary16 rounding (round to nearest, ties to even) of a finite double:
 * 10 fraction bits, exponent range down to 2^-14, subnormal quantum 2^-24;
 * magnitudes that round above 65504 become infinite. */
double nslo_round_f16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  const double a = fabs(x);
  int e;
  frexp(a, &e);            /* a = f 2^e, f in [0.5, 1): a in [2^(e-1), 2^e) */
  int E = e - 1;
  if (E < -14) E = -14;
  const double q = ldexp(1.0, E - 10);
  double r = rint(a / q) * q;   /* the quotient is exact; rint rounds half to even */
  if (r > 65504.0) r = INFINITY;
  return copysign(r, x);
}

/* OCP FP8 E4M3 ("fn": no infinities) rounding, to nearest with ties to even
 * and saturation to the largest finite magnitude: exponent bias 7, 3 fraction
 * bits, normal range [2^-6, 448], subnormal quantum 2^-9. */
double nslo_e4m3_rn(double x) {
  if (x == 0.0 || isnan(x)) return x;
  const double a = fabs(x);
  int e;
  frexp(a, &e);
  int E = e - 1;
  if (E < -6) E = -6;
  const double q = ldexp(1.0, E - 3);
  double r = rint(a / q) * q;
  if (r > 448.0) r = 448.0;
  return copysign(r, x);
}

/* Per-tensor activation scale: the smallest power of two s = 2^k with
 * amax <= 448 s, so quantised x = E4M3(x / s) (an exact scaling) and the
 * dequantisation factor is s; s = 1 for an all-zero tensor.  A power of two
 * keeps the scale, and so every quantisation decision, unchanged under tiny
 * changes of amax.  With amax = f 2^e, f in [0.5, 1): k = e - 9 if f <= 0.875
 * (448 = 0.875 * 2^9), else e - 8. */
static void q8_scales(double amax, float* inv, float* deq) {
  const float a = (float)amax;
  if (a > 0.f) {
    int e;
    const float f = frexpf(a, &e);
    const int k = e - 9 + (f > 0.875f ? 1 : 0);
    *inv = ldexpf(1.0f, -k);
    *deq = ldexpf(1.0f, k);
  } else {
    *inv = 1.0f;
    *deq = 1.0f;
  }
}

/* Quantise a whole tensor (its values are binary16 numbers) with its own amax. */
void nslo_q8_tensor(const double* x, size_t n, double* codes, float* deq) {
  double amax = 0.0;
  for (size_t i = 0; i < n; ++i) amax = fmax(amax, fabs(x[i]));
  float inv;
  q8_scales(amax, &inv, deq);
  for (size_t i = 0; i < n; ++i) {
    const float v = (float)x[i] * inv;          /* exact: inv is a power of two */
    codes[i] = nslo_e4m3_rn((double)v);
  }
}

/* Per-output-channel weight quantisation in binary32: for output channel co,
 * s[co] = max |w| / 448 over the channel's weights, code = E4M3(w / s[co]).
 * Element (co, j) of the channel sits at w[co * so + j * sj] for j < count. */
void nslo_q8_weights(const double* w, int cout, int count, int64_t so, int64_t sj, double* codes,
                     float* s) {
  for (int co = 0; co < cout; ++co) {
    float amax = 0.f;
    for (int j = 0; j < count; ++j) amax = fmaxf(amax, fabsf((float)w[co * so + j * sj]));
    const float sc = amax > 0.f ? amax / 448.0f : 1.0f;
    s[co] = sc;
    for (int j = 0; j < count; ++j) {
      const float v = (float)w[co * so + j * sj] / sc;
      codes[co * so + j * sj] = nslo_e4m3_rn((double)v);
    }
  }
}

/* One FP8 3x3 convolution: input tensor x (binary16 values) quantised with its
 * amax, weights per output channel; the exact sum of code products is scaled
 * by deq * s[co], the bias added, ReLU applied, and the result rounded to
 * binary16 as the stored activation. */
static int conv3_q8(cursor* cur, const double* x, int cin, int H, int W, int cout, double* out) {
  const double* w = take(cur, (int64_t)cout * cin * 9);
  const double* b = take(cur, cout);
  if (!w || !b) return 3;
  const size_t P = (size_t)H * W;
  double* xq = malloc(sizeof(double) * cin * P);
  double* wq = malloc(sizeof(double) * cout * cin * 9);
  double* zb = calloc((size_t)cout, sizeof(double));
  float* s = malloc(sizeof(float) * cout);
  if (!xq || !wq || !zb || !s) { free(xq); free(wq); free(zb); free(s); return 2; }
  float deq;
  nslo_q8_tensor(x, (size_t)cin * P, xq, &deq);
  nslo_q8_weights(w, cout, cin * 9, (int64_t)cin * 9, 1, wq, s);
  nslo_conv2d(xq, cin, H, W, wq, zb, cout, 3, out);
  for (int co = 0; co < cout; ++co) {
    const double f = (double)deq * (double)s[co];
    for (size_t p = 0; p < P; ++p) {
      const double v = out[co * P + p] * f + b[co];
      out[co * P + p] = nslo_round_f16(v > 0.0 ? v : 0.0);
    }
  }
  free(xq); free(wq); free(zb); free(s);
  return 0;
}

/* One FP8 2x2 stride-2 transposed convolution (no activation), same scheme;
 * weights [cin][cout][2][2] quantised per output channel over ci and the four
 * kernel positions. */
static int convT_q8(cursor* cur, const double* x, int cin, int H, int W, int cout, double* out) {
  const double* w = take(cur, (int64_t)cin * cout * 4);
  const double* b = take(cur, cout);
  if (!w || !b) return 3;
  const size_t P = (size_t)H * W, P4 = 4 * P;
  double* xq = malloc(sizeof(double) * cin * P);
  double* wq = malloc(sizeof(double) * cin * cout * 4);
  double* zb = calloc((size_t)cout, sizeof(double));
  float* s = malloc(sizeof(float) * cout);
  if (!xq || !wq || !zb || !s) { free(xq); free(wq); free(zb); free(s); return 2; }
  float deq;
  nslo_q8_tensor(x, (size_t)cin * P, xq, &deq);
  /* output channel co owns the elements ((ci * cout + co) * 4 + k) */
  for (int co = 0; co < cout; ++co) {
    float amax = 0.f;
    for (int ci = 0; ci < cin; ++ci)
      for (int k = 0; k < 4; ++k) amax = fmaxf(amax, fabsf((float)w[((size_t)ci * cout + co) * 4 + k]));
    const float sc = amax > 0.f ? amax / 448.0f : 1.0f;
    s[co] = sc;
    for (int ci = 0; ci < cin; ++ci)
      for (int k = 0; k < 4; ++k) {
        const size_t i = ((size_t)ci * cout + co) * 4 + k;
        wq[i] = nslo_e4m3_rn((double)((float)w[i] / sc));
      }
  }
  nslo_conv_transpose2x2(xq, cin, H, W, wq, zb, cout, out);
  for (int co = 0; co < cout; ++co) {
    const double f = (double)deq * (double)s[co];
    for (size_t p = 0; p < P4; ++p) out[co * P4 + p] = nslo_round_f16(out[co * P4 + p] * f + b[co]);
  }
  free(xq); free(wq); free(zb); free(s);
  return 0;
}

/* The network with FP8 E4M3 convolutions: the first 3x3 convolution (3 input
 * channels) in full precision, every later 3x3 and transposed convolution with
 * per-tensor power-of-two activation scales and per-output-channel weight
 * scales, exact sums of code products, activations stored as binary16 between
 * layers; the adapters in full precision on the binary16 feature map. */
int nslo_net_forward_q8(const double* guide, int H, int W, const double* params, int64_t n_params,
                        int c0, double depth_scale, double* out) {
  if (H % 8 || W % 8 || H <= 0 || W <= 0) return 1;
  cursor cur = {params, n_params};
  const int c1 = c0, c2 = 2 * c0, c3 = 4 * c0, c4 = 8 * c0;
  size_t P0 = (size_t)H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  double* x0 = malloc(sizeof(double) * 3 * P0);
  double* a0 = malloc(sizeof(double) * c1 * P0);
  double* s1 = malloc(sizeof(double) * c1 * P0);
  double* p1 = malloc(sizeof(double) * c1 * P1);
  double* a1 = malloc(sizeof(double) * c2 * P1);
  double* s2 = malloc(sizeof(double) * c2 * P1);
  double* p2 = malloc(sizeof(double) * c2 * P2);
  double* a2 = malloc(sizeof(double) * c3 * P2);
  double* s3 = malloc(sizeof(double) * c3 * P2);
  double* p3 = malloc(sizeof(double) * c3 * P3);
  double* a3 = malloc(sizeof(double) * c4 * P3);
  double* bt = malloc(sizeof(double) * c4 * P3);
  double* cat = malloc(sizeof(double) * 2 * c1 * P0 + sizeof(double) * c4 * P2);
  double* d = malloc(sizeof(double) * c1 * P0 * 2 + sizeof(double) * c4 * P2);
  double* F = malloc(sizeof(double) * c1 * P0);
  double* z = malloc(sizeof(double) * c1 * P0);
  int rc = 0;
  if (!x0 || !a0 || !s1 || !p1 || !a1 || !s2 || !p2 || !a2 || !s3 || !p3 || !a3 || !bt || !cat ||
      !d || !F || !z) { rc = 2; goto done; }

  memcpy(x0, guide, sizeof(double) * 2 * P0);
  for (size_t p = 0; p < P0; ++p) x0[2 * P0 + p] = guide[2 * P0 + p] * depth_scale;

  /* first convolution in full precision, stored as binary16 */
  if ((rc = conv3_relu(&cur, x0, 3, H, W, c1, a0))) goto done;
  for (size_t i = 0; i < (size_t)c1 * P0; ++i) a0[i] = nslo_round_f16(a0[i]);
  /* encoder */
  if ((rc = conv3_q8(&cur, a0, c1, H, W, c1, s1))) goto done;
  nslo_maxpool2(s1, c1, H, W, p1);
  if ((rc = conv3_q8(&cur, p1, c1, H1, W1, c2, a1))) goto done;
  if ((rc = conv3_q8(&cur, a1, c2, H1, W1, c2, s2))) goto done;
  nslo_maxpool2(s2, c2, H1, W1, p2);
  if ((rc = conv3_q8(&cur, p2, c2, H2, W2, c3, a2))) goto done;
  if ((rc = conv3_q8(&cur, a2, c3, H2, W2, c3, s3))) goto done;
  nslo_maxpool2(s3, c3, H2, W2, p3);
  if ((rc = conv3_q8(&cur, p3, c3, H3, W3, c4, a3))) goto done;
  if ((rc = conv3_q8(&cur, a3, c4, H3, W3, c4, bt))) goto done;
  /* decoder: the concatenation (upsampled first, skip second) is one tensor
   * with one activation scale */
  if ((rc = convT_q8(&cur, bt, c4, H3, W3, c3, cat))) goto done;
  memcpy(cat + (size_t)c3 * P2, s3, sizeof(double) * c3 * P2);
  if ((rc = conv3_q8(&cur, cat, 2 * c3, H2, W2, c3, d))) goto done;
  if ((rc = conv3_q8(&cur, d, c3, H2, W2, c3, a2))) goto done;
  if ((rc = convT_q8(&cur, a2, c3, H2, W2, c2, cat))) goto done;
  memcpy(cat + (size_t)c2 * P1, s2, sizeof(double) * c2 * P1);
  if ((rc = conv3_q8(&cur, cat, 2 * c2, H1, W1, c2, d))) goto done;
  if ((rc = conv3_q8(&cur, d, c2, H1, W1, c2, a1))) goto done;
  if ((rc = convT_q8(&cur, a1, c2, H1, W1, c1, cat))) goto done;
  memcpy(cat + (size_t)c1 * P0, s1, sizeof(double) * c1 * P0);
  if ((rc = conv3_q8(&cur, cat, 2 * c1, H, W, c1, d))) goto done;
  if ((rc = conv3_q8(&cur, d, c1, H, W, c1, F))) goto done;
  /* channel adapters on the binary16 feature map */
  if ((rc = adapters_forward(&cur, F, c1, H, W, z, out))) goto done;
  if (cur.left != 0) rc = 4;
done:
  free(x0); free(a0); free(s1); free(p1); free(a1); free(s2); free(p2); free(a2); free(s3);
  free(p3); free(a3); free(bt); free(cat); free(d); free(F); free(z);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Per-layer precision forms of the network (no counterpart in the paper)    */
/* ------------------------------------------------------------------------- */

/* bfloat16 rounding (round to nearest, ties to even) of a finite double:
 * 8 significand bits (7 stored), the binary32 exponent range (normal down to
 * 2^-126, subnormal quantum 2^-133); magnitudes that round above the largest
 * finite value (2 - 2^-7) 2^127 become infinite. */
double nslo_round_bf16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  const double a = fabs(x);
  int e;
  frexp(a, &e);            /* a in [2^(e-1), 2^e) */
  int E = e - 1;
  if (E < -126) E = -126;
  const double q = ldexp(1.0, E - 7);
  double r = rint(a / q) * q;
  if (r > ldexp(2.0 - ldexp(1.0, -7), 127)) r = INFINITY;
  return copysign(r, x);
}

/* Value an activation is stored as after a layer of form `prec`: binary16 for
 * the FP16 form and for the FP8 form (whose activations stay binary16 between
 * layers), bfloat16 for the BF16 form, binary32 for the split-BF16 form, the
 * value itself for FP64. */
static double store_as(int prec, double v) {
  switch (prec) {
    case NSLO_PREC_F16:
    case NSLO_PREC_FP8: return nslo_round_f16(v);
    case NSLO_PREC_BF16: return nslo_round_bf16(v);
    case NSLO_PREC_BF16X3: return (double)(float)v;
    default: return v;
  }
}

/* Operand of a multiplication in a 16-bit form. */
static double operand_as(int prec, double v) {
  return prec == NSLO_PREC_F16 ? nslo_round_f16(v) : (prec == NSLO_PREC_BF16 ? nslo_round_bf16(v) : v);
}

/* One 3x3 (k = 3) or 2x2 stride-2 transposed (k = 2) convolution in form
 * `prec`, weights and bias from the cursor, ReLU after the 3x3 ones:
 *   F64          exact weights and inputs;
 *   F16, BF16    weights and inputs rounded to the 16-bit type, the exact sum
 *                of products plus the bias;
 *   BF16X3       every weight and input split into a bfloat16 high part and
 *                the bfloat16 rounding of the remainder, hi*hi + hi*lo +
 *                lo*hi summed exactly (the lo*lo term dropped) plus the bias;
 *   FP8          the scheme of conv3_q8 / convT_q8.
 * The result is stored as store_as(prec). */
static int conv_prec(cursor* cur, int prec, int k, const double* x, int cin, int H, int W, int cout,
                     double* out) {
  if (prec == NSLO_PREC_FP8)
    return k == 3 ? conv3_q8(cur, x, cin, H, W, cout, out) : convT_q8(cur, x, cin, H, W, cout, out);
  const int64_t nw = (int64_t)cout * cin * (k == 3 ? 9 : 4);
  const double* w = take(cur, nw);
  const double* b = take(cur, cout);
  if (!w || !b) return 3;
  const size_t P = (size_t)H * W, Pout = k == 3 ? P : 4 * P, nx = (size_t)cin * P;
  double* xh = malloc(sizeof(double) * nx);
  double* xl = malloc(sizeof(double) * nx);
  double* wh = malloc(sizeof(double) * nw);
  double* wl = malloc(sizeof(double) * nw);
  double* t = malloc(sizeof(double) * cout * Pout);
  if (!xh || !xl || !wh || !wl || !t) { free(xh); free(xl); free(wh); free(wl); free(t); return 2; }
  const int split = prec == NSLO_PREC_BF16X3;
  for (size_t i = 0; i < nx; ++i) {
    xh[i] = split ? nslo_round_bf16(x[i]) : operand_as(prec, x[i]);
    xl[i] = split ? nslo_round_bf16(x[i] - xh[i]) : 0.0;
  }
  for (int64_t i = 0; i < nw; ++i) {
    wh[i] = split ? nslo_round_bf16(w[i]) : operand_as(prec, w[i]);
    wl[i] = split ? nslo_round_bf16(w[i] - wh[i]) : 0.0;
  }
  if (k == 3) nslo_conv2d(xh, cin, H, W, wh, b, cout, 3, out);
  else nslo_conv_transpose2x2(xh, cin, H, W, wh, b, cout, out);
  if (split) {
    if (k == 3) nslo_conv2d(xh, cin, H, W, wl, NULL, cout, 3, t);
    else nslo_conv_transpose2x2(xh, cin, H, W, wl, NULL, cout, t);
    for (size_t i = 0; i < (size_t)cout * Pout; ++i) out[i] += t[i];
    if (k == 3) nslo_conv2d(xl, cin, H, W, wh, NULL, cout, 3, t);
    else nslo_conv_transpose2x2(xl, cin, H, W, wh, NULL, cout, t);
    for (size_t i = 0; i < (size_t)cout * Pout; ++i) out[i] += t[i];
  }
  for (size_t i = 0; i < (size_t)cout * Pout; ++i) {
    const double v = (k == 3 && out[i] < 0.0) ? 0.0 : out[i];
    out[i] = store_as(prec, v);
  }
  free(xh); free(xl); free(wh); free(wl); free(t);
  return 0;
}

/* One convolution of the network in form `prec` with explicit parameters
 * (conv_prec): k = 3 is a 3x3 convolution followed by ReLU, w [cout][cin][3][3],
 * out [cout][H][W]; k = 2 a 2x2 stride-2 transposed convolution, w
 * [cin][cout][2][2], out [cout][2H][2W]. */
int nslo_conv_layer_prec(int prec, int k, const double* x, int cin, int H, int W, const double* w,
                         const double* b, int cout, double* out) {
  if ((k != 2 && k != 3) || prec < NSLO_PREC_F64 || prec > NSLO_PREC_BF16X3) return 1;
  const int64_t nw = (int64_t)cout * cin * (k == 3 ? 9 : 4);
  double* pb = malloc(sizeof(double) * (size_t)(nw + cout));
  if (!pb) return 2;
  memcpy(pb, w, sizeof(double) * (size_t)nw);
  memcpy(pb + nw, b, sizeof(double) * (size_t)cout);
  cursor cur = {pb, nw + cout};
  const int rc = conv_prec(&cur, prec, k, x, cin, H, W, cout, out);
  free(pb);
  return rc;
}

/* out[i] = the value x[i] is stored as after a layer of form prec. */
void nslo_store_as(int prec, const double* x, size_t n, double* out) {
  for (size_t i = 0; i < n; ++i) out[i] = store_as(prec, x[i]);
}

/* The four channel adapters and their heads on a feature map F [c0][H][W],
 * binary64 (adapters_forward); params: the adapters' part of the blob. */
int nslo_net_adapters(const double* F, int c0, int H, int W, const double* params, int64_t n_params,
                      double* out) {
  cursor cur = {params, n_params};
  double* z = malloc(sizeof(double) * (size_t)c0 * H * W);
  if (!z) return 2;
  int rc = adapters_forward(&cur, F, c0, H, W, z, out);
  if (!rc && cur.left != 0) rc = 4;
  free(z);
  return rc;
}

/* Element count of stored tensor l (0..16, network order) of an H x W image. */
int64_t nslo_net_trace_size(int c0, int H, int W, int l) {
  static const int cmul[17] = {1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1, 1};
  static const int lvl[17] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};
  if (l < 0 || l > 16) return 0;
  return (int64_t)cmul[l] * c0 * (H >> lvl[l]) * (W >> lvl[l]);
}

/* The Sec. 4.3 generator with each of its 17 convolutions in its own
 * precision form: prec[l] for l in network order (0 enc1a, 1 enc1b, 2 enc2a,
 * 3 enc2b, 4 enc3a, 5 enc3b, 6 enc4a, 7 enc4b, 8 up3, 9 dec3a, 10 dec3b,
 * 11 up2, 12 dec2a, 13 dec2b, 14 up1, 15 dec1a, 16 dec1b).  The first
 * convolution (three guide channels) keeps exact weights and inputs whatever
 * its form; its form sets only how its output is stored.  Max-pooling and the
 * skip concatenation act on stored values.  The adapters run in binary64 on the
 * stored feature map F.  trace (nullable): the 17 stored outputs one after
 * another, each planar [C][H_l][W_l] (sizes from nslo_net_trace_size). */
int nslo_net_forward_prec(const double* guide, int H, int W, const double* params, int64_t n_params,
                          int c0, double depth_scale, const int* prec, double* out, double* trace) {
  if (H % 8 || W % 8 || H <= 0 || W <= 0) return 1;
  for (int l = 0; l < 17; ++l)
    if (prec[l] < NSLO_PREC_F64 || prec[l] > NSLO_PREC_BF16X3) return 5;
  cursor cur = {params, n_params};
  const int c1 = c0, c2 = 2 * c0, c3 = 4 * c0, c4 = 8 * c0;
  size_t P0 = (size_t)H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  double* x0 = malloc(sizeof(double) * 3 * P0);
  double* a0 = malloc(sizeof(double) * c1 * P0);
  double* s1 = malloc(sizeof(double) * c1 * P0);
  double* p1 = malloc(sizeof(double) * c1 * P1);
  double* a1 = malloc(sizeof(double) * c2 * P1);
  double* s2 = malloc(sizeof(double) * c2 * P1);
  double* p2 = malloc(sizeof(double) * c2 * P2);
  double* a2 = malloc(sizeof(double) * c3 * P2);
  double* s3 = malloc(sizeof(double) * c3 * P2);
  double* p3 = malloc(sizeof(double) * c3 * P3);
  double* a3 = malloc(sizeof(double) * c4 * P3);
  double* bt = malloc(sizeof(double) * c4 * P3);
  double* cat = malloc(sizeof(double) * 2 * c1 * P0 + sizeof(double) * c4 * P2);
  double* d = malloc(sizeof(double) * c1 * P0 * 2 + sizeof(double) * c4 * P2);
  double* F = malloc(sizeof(double) * c1 * P0);
  double* z = malloc(sizeof(double) * c1 * P0);
  double* tr = trace;
  int rc = 0;
  if (!x0 || !a0 || !s1 || !p1 || !a1 || !s2 || !p2 || !a2 || !s3 || !p3 || !a3 || !bt || !cat ||
      !d || !F || !z) { rc = 2; goto done; }
#define TRACE(buf, n)                                   \
  do {                                                  \
    if (tr) { memcpy(tr, (buf), sizeof(double) * (n)); tr += (n); } \
  } while (0)

  memcpy(x0, guide, sizeof(double) * 2 * P0);
  for (size_t p = 0; p < P0; ++p) x0[2 * P0 + p] = guide[2 * P0 + p] * depth_scale;

  /* first convolution: exact, then stored in its form */
  if ((rc = conv3_relu(&cur, x0, 3, H, W, c1, a0))) goto done;
  for (size_t i = 0; i < (size_t)c1 * P0; ++i) a0[i] = store_as(prec[0], a0[i]);
  TRACE(a0, (size_t)c1 * P0);
  /* encoder */
  if ((rc = conv_prec(&cur, prec[1], 3, a0, c1, H, W, c1, s1))) goto done;
  TRACE(s1, (size_t)c1 * P0);
  nslo_maxpool2(s1, c1, H, W, p1);
  if ((rc = conv_prec(&cur, prec[2], 3, p1, c1, H1, W1, c2, a1))) goto done;
  TRACE(a1, (size_t)c2 * P1);
  if ((rc = conv_prec(&cur, prec[3], 3, a1, c2, H1, W1, c2, s2))) goto done;
  TRACE(s2, (size_t)c2 * P1);
  nslo_maxpool2(s2, c2, H1, W1, p2);
  if ((rc = conv_prec(&cur, prec[4], 3, p2, c2, H2, W2, c3, a2))) goto done;
  TRACE(a2, (size_t)c3 * P2);
  if ((rc = conv_prec(&cur, prec[5], 3, a2, c3, H2, W2, c3, s3))) goto done;
  TRACE(s3, (size_t)c3 * P2);
  nslo_maxpool2(s3, c3, H2, W2, p3);
  if ((rc = conv_prec(&cur, prec[6], 3, p3, c3, H3, W3, c4, a3))) goto done;
  TRACE(a3, (size_t)c4 * P3);
  if ((rc = conv_prec(&cur, prec[7], 3, a3, c4, H3, W3, c4, bt))) goto done;
  TRACE(bt, (size_t)c4 * P3);
  /* decoder: upsampled first, skip second */
  if ((rc = conv_prec(&cur, prec[8], 2, bt, c4, H3, W3, c3, cat))) goto done;
  TRACE(cat, (size_t)c3 * P2);
  memcpy(cat + (size_t)c3 * P2, s3, sizeof(double) * c3 * P2);
  if ((rc = conv_prec(&cur, prec[9], 3, cat, 2 * c3, H2, W2, c3, d))) goto done;
  TRACE(d, (size_t)c3 * P2);
  if ((rc = conv_prec(&cur, prec[10], 3, d, c3, H2, W2, c3, a2))) goto done;
  TRACE(a2, (size_t)c3 * P2);
  if ((rc = conv_prec(&cur, prec[11], 2, a2, c3, H2, W2, c2, cat))) goto done;
  TRACE(cat, (size_t)c2 * P1);
  memcpy(cat + (size_t)c2 * P1, s2, sizeof(double) * c2 * P1);
  if ((rc = conv_prec(&cur, prec[12], 3, cat, 2 * c2, H1, W1, c2, d))) goto done;
  TRACE(d, (size_t)c2 * P1);
  if ((rc = conv_prec(&cur, prec[13], 3, d, c2, H1, W1, c2, a1))) goto done;
  TRACE(a1, (size_t)c2 * P1);
  if ((rc = conv_prec(&cur, prec[14], 2, a1, c2, H1, W1, c1, cat))) goto done;
  TRACE(cat, (size_t)c1 * P0);
  memcpy(cat + (size_t)c1 * P0, s1, sizeof(double) * c1 * P0);
  if ((rc = conv_prec(&cur, prec[15], 3, cat, 2 * c1, H, W, c1, d))) goto done;
  TRACE(d, (size_t)c1 * P0);
  if ((rc = conv_prec(&cur, prec[16], 3, d, c1, H, W, c1, F))) goto done;
  TRACE(F, (size_t)c1 * P0);
#undef TRACE
  /* channel adapters, binary64, on the stored feature map */
  if ((rc = adapters_forward(&cur, F, c1, H, W, z, out))) goto done;
  if (cur.left != 0) rc = 4;
done:
  free(x0); free(a0); free(s1); free(p1); free(a1); free(s2); free(p2); free(a2); free(s3);
  free(p3); free(a3); free(bt); free(cat); free(d); free(F); free(z);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Six-way shading (Sec. 3, directional interpolation)                        */
/* ------------------------------------------------------------------------- */

/* rgb = sum_lights I * sum_{p in x,y,z} |w_p| L_p^{sign w_p} + E, with w the
 * unit toward-light vector in the camera frame (X right, Y up, Z into the
 * screen); A = clamp(1 - T, 0, 1). */
int nslo_shade(const double* lm, int H, int W, const nslo_camera* cam, const nslo_light* lights,
               int n_lights, double* rgba) {
  if (!lm || !cam || !rgba || n_lights < 0 || (n_lights > 0 && !lights)) return 1;
  cam_frame fr;
  cam_setup(cam, &fr);
  size_t P = (size_t)H * W;
  double wts[64][6];
  double inten[64][3];
  if (n_lights > 64) return 1;
  for (int l = 0; l < n_lights; ++l) {
    double v[3] = {lights[l].dir[0], lights[l].dir[1], lights[l].dir[2]};
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nv > 0.0)) return 1;
    for (int k = 0; k < 3; ++k) v[k] /= nv;
    double w[3];
    w[0] = v[0] * fr.r[0] + v[1] * fr.r[1] + v[2] * fr.r[2];
    w[1] = v[0] * fr.u[0] + v[1] * fr.u[1] + v[2] * fr.u[2];
    w[2] = v[0] * fr.f[0] + v[1] * fr.f[1] + v[2] * fr.f[2];
    for (int p = 0; p < 3; ++p) {
      wts[l][2 * p] = w[p] >= 0.0 ? w[p] : 0.0;      /* positive-direction plane */
      wts[l][2 * p + 1] = w[p] < 0.0 ? -w[p] : 0.0;  /* negative-direction plane */
    }
    for (int c = 0; c < 3; ++c) inten[l][c] = lights[l].intensity[c];
  }
  for (size_t p = 0; p < P; ++p) {
    double E = lm[7 * P + p];
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int l = 0; l < n_lights; ++l) {
        double s = 0.0;
        for (int q = 0; q < 6; ++q) s += wts[l][q] * lm[q * P + p];
        acc += inten[l][c] * s;
      }
      rgba[c * P + p] = acc + E;
    }
    double a = 1.0 - lm[6 * P + p];
    rgba[3 * P + p] = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Obstacle shadowing (Sec. 4.5): the smoke shell depth D of the guide moved   */
/* into the light's frame and compared with a shadow map of the obstacle.     */
/* ------------------------------------------------------------------------- */

/* Light frame of a directional light, built in binary64 and rounded once to
 * binary32: w = -dir/|dir| (the propagation direction), e1 = normalize(w x a)
 * with a = +Y, or +Z when |w_y| > 0.9, e2 = e1 x w.  The map is the square of
 * side S = |(nx, ny, nz)| centred on the grid centre c, in the plane through c
 * spanned by (e1, e2). */
typedef struct {
  float w[3], e1[3], e2[3], c[3], S;
} light_frame;

static int light_setup(const float dir[3], int nx, int ny, int nz, light_frame* L) {
  double v[3] = {dir[0], dir[1], dir[2]};
  double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  if (!(nv > 0.0)) return 1;
  double w[3] = {-v[0] / nv, -v[1] / nv, -v[2] / nv};
  double a[3] = {0.0, 1.0, 0.0};
  if (fabs(w[1]) > 0.9) { a[1] = 0.0; a[2] = 1.0; }
  double e1[3] = {w[1] * a[2] - w[2] * a[1], w[2] * a[0] - w[0] * a[2], w[0] * a[1] - w[1] * a[0]};
  double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int k = 0; k < 3; ++k) e1[k] /= l1;
  double e2[3] = {e1[1] * w[2] - e1[2] * w[1], e1[2] * w[0] - e1[0] * w[2], e1[0] * w[1] - e1[1] * w[0]};
  for (int k = 0; k < 3; ++k) {
    L->w[k] = (float)w[k];
    L->e1[k] = (float)e1[k];
    L->e2[k] = (float)e2[k];
  }
  L->c[0] = (float)nx * 0.5f;
  L->c[1] = (float)ny * 0.5f;
  L->c[2] = (float)nz * 0.5f;
  L->S = (float)sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
  return 0;
}

/* Slab test of the unit voxel with low corner (i, j, k) against the line
 * o + t w (t unbounded); returns 1 and the entry parameter on a hit (touching
 * counts). */
static int voxel_entry(const float o[3], const float w[3], int i, int j, int k, float* t_enter) {
  const float lo[3] = {(float)i, (float)j, (float)k};
  float tn = -INFINITY, tf = INFINITY;
  for (int q = 0; q < 3; ++q) {
    const float hi = lo[q] + 1.0f;
    if (w[q] != 0.0f) {
      float ta = (lo[q] - o[q]) / w[q];
      float tb = (hi - o[q]) / w[q];
      float nr = ta < tb ? ta : tb;
      float fr = ta < tb ? tb : ta;
      if (nr > tn) tn = nr;
      if (fr < tf) tf = fr;
    } else if (o[q] < lo[q] || o[q] > hi) {
      return 0;
    }
  }
  if (!(tn <= tf)) return 0;
  *t_enter = tn;
  return 1;
}

/* Shadow map of the obstacle mask for one directional light: texel (i, j)
 * (column i, row j of an R x R map) holds the entry parameter t of the first
 * occupied voxel along the line o + t w through
 *   o = c + a e1 + b e2,  a = ((i + 0.5)/R - 0.5) S,  b = ((j + 0.5)/R - 0.5) S,
 * i.e. the minimum over all occupied voxels the line meets (brute force), or
 * +infinity.  t is signed distance from the map plane along w. */
int nslo_shadow_map(const uint8_t* mask, int nx, int ny, int nz, const float dir[3], int R,
                    float* out) {
  if (!mask || !dir || !out || R < 1) return 1;
  light_frame L;
  if (light_setup(dir, nx, ny, nz, &L)) return 1;
  const size_t nvox = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < R; ++j) {
    for (int i = 0; i < R; ++i) {
      float ua = ((float)i + 0.5f) / (float)R;
      float ub = ((float)j + 0.5f) / (float)R;
      float a = (ua - 0.5f) * L.S;
      float b = (ub - 0.5f) * L.S;
      float o[3];
      for (int k = 0; k < 3; ++k) {
        float t1 = a * L.e1[k];
        float t2 = b * L.e2[k];
        o[k] = (L.c[k] + t1) + t2;
      }
      float best = INFINITY;
      for (size_t v = 0; v < nvox; ++v) {
        if (!mask[v]) continue;
        const int vi = (int)(v % nx), vj = (int)((v / nx) % ny), vk = (int)(v / ((size_t)nx * ny));
        float te;
        if (voxel_entry(o, L.w, vi, vj, vk, &te) && te < best) best = te;
      }
      out[(size_t)j * R + i] = best;
    }
  }
  return 0;
}

/* Visibility of pixel p's smoke shell from light l: the shell point is
 * x = o + (t_in + D) d on the pixel's ray (t_in its box entry, D the guide's
 * depth channel; the jitter offset below one step is ignored); in the light's
 * frame, relative to c, it has map coordinates (a, b) = (x - c).(e1, e2) and
 * depth z = (x - c).w, all in binary32 in this order.  It is shadowed when its
 * texel (floor((a/S + 1/2) R), likewise for b) lies on the map and
 * z > t_hit + bias.  D = 0 (no shell) and rays missing the box are lit. */
static int shell_shadowed(const cam_frame* fr, const float nbox[3], const light_frame* L,
                          const float* map, int R, float bias, int i, int j, float D) {
  if (!(D > 0.0f) || !map) return 0;
  float o[3], d[3], tin, tout;
  pixel_ray(fr, i, j, o, d);
  if (!clip_box(o, d, nbox, &tin, &tout)) return 0;
  const float t = tin + D;
  float rel[3];
  for (int k = 0; k < 3; ++k) {
    float st = t * d[k];
    float x = o[k] + st;
    rel[k] = x - L->c[k];
  }
  float pa0 = rel[0] * L->e1[0], pa1 = rel[1] * L->e1[1], pa2 = rel[2] * L->e1[2];
  float pb0 = rel[0] * L->e2[0], pb1 = rel[1] * L->e2[1], pb2 = rel[2] * L->e2[2];
  float pz0 = rel[0] * L->w[0], pz1 = rel[1] * L->w[1], pz2 = rel[2] * L->w[2];
  float a = (pa0 + pa1) + pa2;
  float b = (pb0 + pb1) + pb2;
  float z = (pz0 + pz1) + pz2;
  float fa = (a / L->S + 0.5f) * (float)R;
  float fb = (b / L->S + 0.5f) * (float)R;
  float ffa = floorf(fa), ffb = floorf(fb);
  if (!(ffa >= 0.0f && ffa < (float)R && ffb >= 0.0f && ffb < (float)R)) return 0;
  const float th = map[(size_t)(int)ffb * R + (int)ffa];
  const float lim = th + bias;
  return z > lim;
}

/* Six-way shading with obstacle shadows: nslo_shade with each light's term
 * multiplied by its visibility (0 or 1); maps[l] may be NULL (no obstacle
 * shadow for light l).  guide is the float32 [3][H][W] guide (D = plane 2). */
int nslo_shade_shadowed(const double* lm, const float* guide, int H, int W, const nslo_camera* cam,
                        const nslo_light* lights, int n_lights, int nx, int ny, int nz,
                        const float* const* maps, int R, float bias, double* rgba) {
  if (!lm || !guide || !cam || !rgba || n_lights < 0 || n_lights > 64 || (n_lights > 0 && !lights))
    return 1;
  cam_frame fr;
  cam_setup(cam, &fr);
  const float nbox[3] = {(float)nx, (float)ny, (float)nz};
  const size_t P = (size_t)H * W;
  double wts[64][6];
  light_frame LF[64];
  for (int l = 0; l < n_lights; ++l) {
    double v[3] = {lights[l].dir[0], lights[l].dir[1], lights[l].dir[2]};
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nv > 0.0)) return 1;
    for (int k = 0; k < 3; ++k) v[k] /= nv;
    double w[3];
    w[0] = v[0] * fr.r[0] + v[1] * fr.r[1] + v[2] * fr.r[2];
    w[1] = v[0] * fr.u[0] + v[1] * fr.u[1] + v[2] * fr.u[2];
    w[2] = v[0] * fr.f[0] + v[1] * fr.f[1] + v[2] * fr.f[2];
    for (int p = 0; p < 3; ++p) {
      wts[l][2 * p] = w[p] >= 0.0 ? w[p] : 0.0;
      wts[l][2 * p + 1] = w[p] < 0.0 ? -w[p] : 0.0;
    }
    if (light_setup(lights[l].dir, nx, ny, nz, &LF[l])) return 1;
  }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      const size_t p = (size_t)j * W + i;
      const float D = guide[2 * P + p];
      double vis[64];
      for (int l = 0; l < n_lights; ++l)
        vis[l] = shell_shadowed(&fr, nbox, &LF[l], maps ? maps[l] : NULL, R, bias, i, j, D) ? 0.0 : 1.0;
      const double E = lm[7 * P + p];
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int l = 0; l < n_lights; ++l) {
          double s = 0.0;
          for (int q = 0; q < 6; ++q) s += wts[l][q] * lm[q * P + p];
          acc += vis[l] * lights[l].intensity[c] * s;
        }
        rgba[c * P + p] = acc + E;
      }
      double a = 1.0 - lm[6 * P + p];
      rgba[3 * P + p] = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
    }
  return 0;
}
