/*
 * a3fr_oracle.c -- plain CPU oracle of the foveated 3D Gaussian Splatting forward
 * rasterizer (A3FR, Sec. 2.3 "Neural Rendering", Sec. 3.4 "AMR-based Rendering Strategy",
 * Sec. 3.5 "Implementation Details", Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or execute
 * this file: it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark can check the CUDA path against a slow, obviously correct restatement
 * of the method.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it computes, in the paper's order (projection -> per-tile depth sort ->
 * front-to-back volume rendering, Sec. 2.3), written as the plain definition:
 *   - per Gaussian: activation, camera transform, EWA covariance, conic, 3-sigma
 *     radius, tile rectangle, SH colour;
 *   - the 64-bit (tile << 32 | depth bits) keys in Gaussian order, sorted with a
 *     stable comparison sort (library qsort with the emission position as tie-break);
 *   - per-tile [start, end) ranges of the sorted keys;
 *   - the tile accuracy levels of Eq. 1 / Sec. 3.4 from the gaze;
 *   - for every rendered pixel a walk over ONE global list of the visible Gaussians
 *     sorted by (depth bits, index) -- no tiles, no blocking -- skipping Gaussians
 *     whose tile rectangle does not contain the pixel's tile;
 *   - the un-rendered pixels of a 2x2 block inherit its top-left pixel (Sec. 3.4).
 *
 * Precision: the configurations fix fp32, and the integer results (depth bits, tile
 * rectangles) are decided by fp32 arithmetic, so the projection runs in fp32 with a
 * fixed operation order and no contraction (build with -ffp-contract=off).  The one
 * transcendental on that path, exp, is the project's own Cody-Waite + Taylor exp
 * (or_exp below), so both sides can round it identically.  The per-pixel exp of the
 * Gaussian falloff is the correctly rounded fp32 value of the fp64 exp, and the
 * oracle reports each pixel's smallest relative margin to the two thresholds that
 * an ulp-level difference there can flip (alpha >= 1/255 and T >= 1e-4).
 *
 * Readings where the paper is silent (it cites the original 3DGS renderer for all
 * constants): near plane 0.2, 0.3 px^2 low-pass, radius ceil(3 sqrt(lambda_max))
 * with an eigenvalue floor of 0.1, alpha clamp 0.99, skip alpha < 1/255, stop when
 * T would drop below 1e-4, colour = max(0, SH + 0.5), background 0, Jacobian
 * clamp 1.3 tan(fov/2), pixel (i, j) sampled at (i, j).  Tile rectangle:
 * [floor((u - r) / B), floor((u + r) / B) + 1) clamped to the grid.  Level labels
 * of a 2x2 block: top-left 1, bottom-right 2, top-right 3, bottom-left 4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy, znear;
  float world_to_cam[12]; /* row-major 3x4 [R | t] */
} or_camera;

typedef struct {
  int32_t n_layers;       /* 1..4 */
  float theta_deg[3];     /* eccentricity boundary of layer k, k < n_layers - 1 */
  float dtheta_deg;       /* tracking-error margin of Eq. 1 */
  int32_t level[4];       /* pixel-density level (1..4) of layer k */
} or_fovea;

/* ---------------------------------------------------------------- exp (key path)
 * Cody-Waite argument reduction x = k ln2 + r, |r| <= ln2 / 2, with ln2 split into
 * a 16-bit head (45426 / 2^16, so k * head is exact for |k| < 2^8) and an fp32 tail,
 * then the degree-7 Taylor polynomial of e^r in Horner form (separately rounded
 * multiplies and adds), then an exact scaling by 2^k built from the exponent field.
 * Arguments are clamped to [-87, 88] so 2^k stays a normal number. */
static const float OR_INV_LN2 = 0x1.715476p+0f;   /* fp32(1 / ln 2) */
static const float OR_LN2_HI = 0x1.62e4p-1f;      /* 45426 / 65536 */
static const float OR_LN2_LO = 0x1.7f7d1cp-20f;   /* fp32(ln 2 - 45426 / 65536) */
static const float OR_INV_FACT[8] = {             /* fp32(1 / n!) */
    0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f,
    0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f};

float or_exp(float x) {
  if (x > 88.0f) x = 88.0f;
  if (x < -87.0f) x = -87.0f;
  float k = rintf(x * OR_INV_LN2);
  float r = (x - k * OR_LN2_HI) - k * OR_LN2_LO;
  float p = OR_INV_FACT[7];
  for (int i = 6; i >= 0; --i) p = p * r + OR_INV_FACT[i];
  int32_t ki = (int32_t)k;
  uint32_t bits = (uint32_t)(ki + 127) << 23;
  float scale;
  memcpy(&scale, &bits, sizeof scale);
  return p * scale;
}

/* ------------------------------------------------------- real SH basis, 3DGS order
 * Coefficient k = l^2 + l + m of degree l <= 3 multiplies the real spherical
 * harmonic of (l, m) evaluated at the unit view direction d = (x, y, z), with the
 * sign convention of the original 3DGS renderer.  The normalisations are the
 * closed forms sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0)
 * multiplied out for each polynomial. */
void or_sh_basis(const float d[3], int degree, float *out) {
  const double PI = 3.14159265358979323846;
  const float x = d[0], y = d[1], z = d[2];
  out[0] = (float)(0.5 * sqrt(1.0 / PI));
  if (degree < 1) return;
  const float c1 = (float)sqrt(3.0 / (4.0 * PI));
  out[1] = -c1 * y;
  out[2] = c1 * z;
  out[3] = -c1 * x;
  if (degree < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  const float c2a = (float)(0.5 * sqrt(15.0 / PI));
  const float c2b = (float)(0.25 * sqrt(5.0 / PI));
  const float c2c = (float)(0.25 * sqrt(15.0 / PI));
  out[4] = c2a * (x * y);
  out[5] = -c2a * (y * z);
  out[6] = c2b * (2.0f * zz - xx - yy);
  out[7] = -c2a * (x * z);
  out[8] = c2c * (xx - yy);
  if (degree < 3) return;
  const float c3a = (float)(0.25 * sqrt(35.0 / (2.0 * PI)));
  const float c3b = (float)(0.5 * sqrt(105.0 / PI));
  const float c3c = (float)(0.25 * sqrt(21.0 / (2.0 * PI)));
  const float c3d = (float)(0.25 * sqrt(7.0 / PI));
  const float c3e = (float)(0.25 * sqrt(105.0 / PI));
  out[9] = -c3a * (y * (3.0f * xx - yy));
  out[10] = c3b * (x * y * z);
  out[11] = -c3c * (y * (4.0f * zz - xx - yy));
  out[12] = c3d * (z * (2.0f * zz - 3.0f * xx - 3.0f * yy));
  out[13] = -c3c * (x * (4.0f * zz - xx - yy));
  out[14] = c3e * (z * (xx - yy));
  out[15] = -c3a * (x * (xx - 3.0f * yy));
}

/* ------------------------------------------------------------- per-Gaussian step
 * Record layout (12 floats): u, v, conic a, conic b, conic c, opacity, r, g, b,
 * depth, radius, visible.  Rect: x0, y0, x1, y1 (tiles, half-open). */
enum { OR_REC = 12 };

static void or_project_one(int i, int degree, const float *means, const float *log_scales,
                           const float *quats, const float *opacity_logits, const float *sh,
                           const or_camera *cam, int tile, int tiles_x, int tiles_y,
                           float *rec, int32_t *rect, uint32_t *touched) {
  float *o = rec + (size_t)i * OR_REC;
  int32_t *rc = rect + (size_t)i * 4;
  memset(o, 0, sizeof(float) * OR_REC);
  rc[0] = rc[1] = rc[2] = rc[3] = 0;
  touched[i] = 0;

  const float *W = cam->world_to_cam;
  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  /* camera-space position t = R mu + t_c (Sec. 2.3, projection) */
  const float tx = ((W[0] * mx + W[1] * my) + W[2] * mz) + W[3];
  const float ty = ((W[4] * mx + W[5] * my) + W[6] * mz) + W[7];
  const float tz = ((W[8] * mx + W[9] * my) + W[10] * mz) + W[11];
  if (!(tz > cam->znear)) return;

  /* activation: scale = exp(log scale), unit quaternion */
  float s2[3];
  for (int j = 0; j < 3; ++j) {
    const float s = or_exp(log_scales[3 * i + j]);
    s2[j] = s * s;
  }
  float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
  const float qn = sqrtf(((qw * qw + qx * qx) + qy * qy) + qz * qz);
  qw = qw / qn; qx = qx / qn; qy = qy / qn; qz = qz / qn;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  R[0][1] = 2.0f * (qx * qy - qw * qz);
  R[0][2] = 2.0f * (qx * qz + qw * qy);
  R[1][0] = 2.0f * (qx * qy + qw * qz);
  R[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
  R[1][2] = 2.0f * (qy * qz - qw * qx);
  R[2][0] = 2.0f * (qx * qz - qw * qy);
  R[2][1] = 2.0f * (qy * qz + qw * qx);
  R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);

  /* 3D covariance Sigma = R diag(s^2) R^T */
  float S[3][3];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k)
      S[j][k] = ((R[j][0] * s2[0]) * R[k][0] + (R[j][1] * s2[1]) * R[k][1]) + (R[j][2] * s2[2]) * R[k][2];

  /* EWA: Jacobian of the pinhole projection at the (clamped) camera-space point */
  const float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
  const float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
  const float txz = tx / tz, tyz = ty / tz;
  const float xc = fminf(limx, fmaxf(-limx, txz)) * tz;
  const float yc = fminf(limy, fmaxf(-limy, tyz)) * tz;
  const float tz2 = tz * tz;
  const float J00 = cam->fx / tz, J02 = -(cam->fx * xc) / tz2;
  const float J11 = cam->fy / tz, J12 = -(cam->fy * yc) / tz2;
  /* T = J W (W = camera rotation), a 2x3 matrix; J01 = J10 = 0 */
  float T[2][3];
  for (int j = 0; j < 3; ++j) {
    T[0][j] = J00 * W[0 + j] + J02 * W[8 + j];
    T[1][j] = J11 * W[4 + j] + J12 * W[8 + j];
  }
  /* Sigma' = T Sigma T^T via U = T Sigma */
  float U[2][3];
  for (int r = 0; r < 2; ++r)
    for (int l = 0; l < 3; ++l)
      U[r][l] = (T[r][0] * S[0][l] + T[r][1] * S[1][l]) + T[r][2] * S[2][l];
  const float c00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2];
  const float c01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
  const float c11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2];
  const float a = c00 + 0.3f, b = c01, c = c11 + 0.3f;   /* low-pass filter */
  const float det = a * c - b * b;
  if (!(det > 0.0f)) return;
  const float mid = 0.5f * (a + c);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
  const float radius = ceilf(3.0f * sqrtf(lam));
  const float u = cam->fx * txz + cam->cx;
  const float v = cam->fy * tyz + cam->cy;

  /* tile rectangle of the 3-sigma square, half-open, clamped to the grid */
  const float fb = (float)tile;
  const float fx0 = fminf((float)tiles_x, fmaxf(0.0f, floorf((u - radius) / fb)));
  const float fx1 = fminf((float)tiles_x, fmaxf(0.0f, floorf((u + radius) / fb) + 1.0f));
  const float fy0 = fminf((float)tiles_y, fmaxf(0.0f, floorf((v - radius) / fb)));
  const float fy1 = fminf((float)tiles_y, fmaxf(0.0f, floorf((v + radius) / fb) + 1.0f));
  const int32_t x0 = (int32_t)fx0, x1 = (int32_t)fx1, y0 = (int32_t)fy0, y1 = (int32_t)fy1;
  if (x0 >= x1 || y0 >= y1) return;

  /* opacity = sigmoid(logit) */
  const float opacity = 1.0f / (1.0f + or_exp(-opacity_logits[i]));

  /* colour: SH along the unit direction from the camera centre to the mean */
  float C[3];
  for (int j = 0; j < 3; ++j) C[j] = -((W[0 + j] * W[3] + W[4 + j] * W[7]) + W[8 + j] * W[11]);
  float d[3] = {mx - C[0], my - C[1], mz - C[2]};
  const float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  d[0] /= dn; d[1] /= dn; d[2] /= dn;
  float basis[16];
  or_sh_basis(d, degree, basis);
  const int K = (degree + 1) * (degree + 1);
  const float *coef = sh + (size_t)i * K * 3;
  float rgb[3];
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.0f;
    for (int k = 0; k < K; ++k) acc += basis[k] * coef[3 * k + ch];
    rgb[ch] = fmaxf(0.0f, acc + 0.5f);
  }

  const float inv = 1.0f / det;
  o[0] = u; o[1] = v;
  o[2] = c * inv; o[3] = -b * inv; o[4] = a * inv;
  o[5] = opacity;
  o[6] = rgb[0]; o[7] = rgb[1]; o[8] = rgb[2];
  o[9] = tz; o[10] = radius; o[11] = 1.0f;
  rc[0] = x0; rc[1] = y0; rc[2] = x1; rc[3] = y1;
  touched[i] = (uint32_t)((x1 - x0) * (y1 - y0));
}

static int or_tiles(int extent, int tile) { return (extent + tile - 1) / tile; }

void or_preprocess(int n, int degree, const float *means, const float *log_scales,
                   const float *quats, const float *opacity_logits, const float *sh,
                   const or_camera *cam, int tile, float *rec, int32_t *rect,
                   uint32_t *touched) {
  const int tiles_x = or_tiles(cam->width, tile), tiles_y = or_tiles(cam->height, tile);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    or_project_one(i, degree, means, log_scales, quats, opacity_logits, sh, cam, tile,
                   tiles_x, tiles_y, rec, rect, touched);
}

/* ------------------------------------------------------------- keys and ranges */
typedef struct { uint64_t key; uint64_t pos; uint32_t val; } or_pair;

static int or_cmp_pair(const void *pa, const void *pb) {
  const or_pair *a = (const or_pair *)pa, *b = (const or_pair *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->pos < b->pos ? -1 : (a->pos > b->pos ? 1 : 0);
}

static uint32_t or_float_bits(float f) { uint32_t u; memcpy(&u, &f, sizeof u); return u; }

/* Emit one (tile << 32 | depth bits, Gaussian index) pair per touched tile, Gaussians
 * in index order and tiles row-major, then sort stably by key.  Returns the count. */
int64_t or_sorted_keys(int n, const float *rec, const int32_t *rect, int tiles_x,
                       uint64_t *keys, uint32_t *vals) {
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t *rc = rect + (size_t)i * 4;
    if (rec[(size_t)i * OR_REC + 11] == 0.0f) continue;
    total += (int64_t)(rc[2] - rc[0]) * (rc[3] - rc[1]);
  }
  if (keys == NULL) return total;
  or_pair *p = (or_pair *)malloc(sizeof(or_pair) * (size_t)(total > 0 ? total : 1));
  int64_t w = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t *rc = rect + (size_t)i * 4;
    if (rec[(size_t)i * OR_REC + 11] == 0.0f) continue;
    const uint64_t db = or_float_bits(rec[(size_t)i * OR_REC + 9]);
    for (int ty = rc[1]; ty < rc[3]; ++ty)
      for (int tx = rc[0]; tx < rc[2]; ++tx) {
        p[w].key = ((uint64_t)(ty * tiles_x + tx) << 32) | db;
        p[w].pos = (uint64_t)w;
        p[w].val = (uint32_t)i;
        ++w;
      }
  }
  qsort(p, (size_t)total, sizeof(or_pair), or_cmp_pair);
  for (int64_t j = 0; j < total; ++j) { keys[j] = p[j].key; vals[j] = p[j].val; }
  free(p);
  return total;
}

void or_tile_ranges(int64_t count, const uint64_t *keys, int n_tiles, uint32_t *ranges) {
  memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles);
  for (int64_t j = 0; j < count; ++j) {
    const uint32_t t = (uint32_t)(keys[j] >> 32);
    if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[2 * t] = (uint32_t)j;
    if (j == count - 1 || (uint32_t)(keys[j + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
  }
}

/* --------------------------------------------------------- foveation (Eq. 1, AMR)
 * r_k = f tan(theta_k + dtheta) (Eq. 1 with rho d = f in pixels); a tile's distance
 * to the gaze is the distance from the gaze to the nearest pixel centre of the tile.
 * The tile takes the level of the innermost layer whose radius reaches it. */
void or_layer_radii2(const or_camera *cam, const or_fovea *fv, float *r2) {
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < 3; ++k) {
    const float r = (float)((double)cam->fx * tan(((double)fv->theta_deg[k] + (double)fv->dtheta_deg) * PI / 180.0));
    r2[k] = r * r;
  }
}

void or_level_map(const or_camera *cam, int tile, const or_fovea *fv, const float gaze[2],
                  uint8_t *level) {
  const int tiles_x = or_tiles(cam->width, tile), tiles_y = or_tiles(cam->height, tile);
  float r2[3];
  or_layer_radii2(cam, fv, r2);
  for (int ty = 0; ty < tiles_y; ++ty)
    for (int tx = 0; tx < tiles_x; ++tx) {
      const float x0 = (float)(tx * tile), y0 = (float)(ty * tile);
      const float x1 = (float)((tx + 1) * tile < cam->width ? (tx + 1) * tile - 1 : cam->width - 1);
      const float y1 = (float)((ty + 1) * tile < cam->height ? (ty + 1) * tile - 1 : cam->height - 1);
      const float dx = fmaxf(fmaxf(x0 - gaze[0], gaze[0] - x1), 0.0f);
      const float dy = fmaxf(fmaxf(y0 - gaze[1], gaze[1] - y1), 0.0f);
      const float d2 = dx * dx + dy * dy;
      int layer = fv->n_layers - 1;
      for (int k = 0; k < fv->n_layers - 1; ++k)
        if (d2 <= r2[k]) { layer = k; break; }
      level[ty * tiles_x + tx] = (uint8_t)fv->level[layer];
    }
}

/* label of pixel (x, y) inside its 2x2 block: TL 1, BR 2, TR 3, BL 4 */
static int or_label(int x, int y) {
  static const int L[2][2] = {{1, 4}, {3, 2}}; /* [x & 1][y & 1] */
  return L[x & 1][y & 1];
}

/* ------------------------------------------------------------------- compositing */
typedef struct { uint32_t depth_bits; uint32_t idx; } or_order;

/* One entry of the global depth-ordered list as the per-pixel walk reads it: the
 * Gaussian's index and a copy of its tile rectangle, so that the walk reads the list
 * front to back instead of looking each rectangle up by index (the same list, the same
 * tests, in the same order). */
typedef struct { uint16_t x0, y0, x1, y1; uint32_t idx; } or_entry;   /* tiles < 2^16 */

static int or_cmp_order(const void *pa, const void *pb) {
  const or_order *a = (const or_order *)pa, *b = (const or_order *)pb;
  if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Front-to-back volume rendering of one pixel over the global depth-sorted list.
 *
 * Two decisions per Gaussian can be flipped by an ulp-level difference in the falloff exp:
 * the skip of alpha < 1/255 and the stop before a Gaussian that would bring T below 1e-4.
 * The walk records, as the pixel's margin, the smallest relative distance of any such
 * decision to its threshold (|255 raw - 1| for the skip, |10^4 T' - 1| for the stop) and
 * where it was taken (position in the list and kind).  flip_j >= 0 re-runs the walk with
 * the decision of kind flip_kind at list position flip_j taken the other way and every
 * other decision as usual: the image a renderer would produce if only that decision
 * flipped. */
enum { OR_FLIP_NONE = -1, OR_FLIP_SKIP = 0, OR_FLIP_STOP = 1 };

typedef struct {
  float rgb[3], t_final, margin, depth;
  int32_t n_contrib, n_eval, n_blend;
  int32_t min_j, min_kind;   /* where the smallest margin was taken */
} or_walk_result;

static void or_walk(int x, int y, int tile, const float *rec, const int32_t *rect,
                    const or_entry *list, int n_vis, int flip_j, int flip_kind,
                    or_walk_result *res) {
  const int ptx = x / tile, pty = y / tile;
  float T = 1.0f, C[3] = {0.0f, 0.0f, 0.0f};
  float Z = 0.0f;   /* expected depth: the blend weights applied to camera-space depth */
  int32_t contrib = 0, evals = 0, blends = 0;
  float m = INFINITY;
  int32_t min_j = -1, min_kind = OR_FLIP_NONE;
  for (int j = 0; j < n_vis; ++j) {
    const or_entry *le = list + j;
    /* the pixel's tile inside the rectangle (one combined test, no short circuit) */
    if (!((ptx >= le->x0) & (ptx < le->x1) & (pty >= le->y0) & (pty < le->y1))) continue;
    const uint32_t g = le->idx;
    const float *o = rec + (size_t)g * OR_REC;
    ++evals;
    const float dx = o[0] - (float)x, dy = o[1] - (float)y;
    const float power = -0.5f * (o[2] * dx * dx + o[4] * dy * dy) - o[3] * dx * dy;
    if (power > 0.0f) continue;
    const float raw = o[5] * (float)exp((double)power);
    const float ma = fabsf(raw - (1.0f / 255.0f)) * 255.0f;
    if (ma < m) { m = ma; min_j = j; min_kind = OR_FLIP_SKIP; }
    const float alpha = fminf(0.99f, raw);
    int skip = alpha < 1.0f / 255.0f;
    if (j == flip_j && flip_kind == OR_FLIP_SKIP) skip = !skip;
    if (skip) continue;
    const float testT = T * (1.0f - alpha);
    const float mt = fabsf(testT - 0.0001f) * 10000.0f;
    if (mt < m) { m = mt; min_j = j; min_kind = OR_FLIP_STOP; }
    int stop = testT < 0.0001f;
    if (j == flip_j && flip_kind == OR_FLIP_STOP) stop = !stop;
    if (stop) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += o[6 + ch] * alpha * T;
    Z += o[9] * alpha * T;
    T = testT;
    contrib = evals;
    ++blends;
  }
  res->rgb[0] = C[0]; res->rgb[1] = C[1]; res->rgb[2] = C[2];   /* + T * background, 0 */
  res->t_final = T;
  res->n_contrib = contrib;
  res->n_eval = evals;
  res->n_blend = blends;
  res->margin = m;
  res->depth = Z;
  res->min_j = min_j;
  res->min_kind = min_kind;
}

/* Pixels whose margin is below this also get the image with their nearest decision
 * flipped (rgb_alt); the others get rgb_alt = rgb. */
static const float OR_ALT_BELOW = 1e-3f;

static void or_shade(int x, int y, int tile, const float *rec, const int32_t *rect,
                     const or_entry *list, int n_vis, float out[3], float *t_final,
                     int32_t *n_contrib, int32_t *n_eval, float *margin, float *depth,
                     float *out_alt, int32_t *n_blend) {
  or_walk_result r;
  or_walk(x, y, tile, rec, rect, list, n_vis, -1, OR_FLIP_NONE, &r);
  out[0] = r.rgb[0]; out[1] = r.rgb[1]; out[2] = r.rgb[2];
  *t_final = r.t_final;
  *n_contrib = r.n_contrib;
  *n_eval = r.n_eval;
  *margin = r.margin;
  if (depth) *depth = r.depth;
  if (n_blend) *n_blend = r.n_blend;
  if (out_alt) {
    out_alt[0] = r.rgb[0]; out_alt[1] = r.rgb[1]; out_alt[2] = r.rgb[2];
    if (r.min_j >= 0 && r.margin < OR_ALT_BELOW) {
      or_walk_result a;
      or_walk(x, y, tile, rec, rect, list, n_vis, r.min_j, r.min_kind, &a);
      out_alt[0] = a.rgb[0]; out_alt[1] = a.rgb[1]; out_alt[2] = a.rgb[2];
    }
  }
}

static or_entry *or_global_list(int n, const float *rec, const int32_t *rect, int *n_vis) {
  or_order *order = (or_order *)malloc(sizeof(or_order) * (size_t)(n > 0 ? n : 1));
  int c = 0;
  for (int i = 0; i < n; ++i)
    if (rec[(size_t)i * OR_REC + 11] != 0.0f) {
      order[c].depth_bits = or_float_bits(rec[(size_t)i * OR_REC + 9]);
      order[c].idx = (uint32_t)i;
      ++c;
    }
  qsort(order, (size_t)c, sizeof(or_order), or_cmp_order);
  or_entry *list = (or_entry *)malloc(sizeof(or_entry) * (size_t)(c > 0 ? c : 1));
  for (int j = 0; j < c; ++j) {
    const int32_t *rc = rect + (size_t)order[j].idx * 4;
    list[j].x0 = (uint16_t)rc[0]; list[j].y0 = (uint16_t)rc[1];
    list[j].x1 = (uint16_t)rc[2]; list[j].y1 = (uint16_t)rc[3];
    list[j].idx = order[j].idx;
  }
  free(order);
  *n_vis = c;
  return list;
}

/* Render pixels.  level == NULL renders every pixel (full resolution); otherwise a
 * pixel is rendered iff its 2x2 label <= its tile's level and every other pixel takes
 * the value of its block's top-left pixel.  pix == NULL means all W*H pixels in
 * row-major order; otherwise the n_pix (x, y) pairs listed.  Per output pixel:
 * rgb[3], T_final, n_contrib, n_eval and the threshold margin of the pixel that was
 * actually shaded (the top-left one for inherited pixels); rendered[] is 1 when the
 * pixel itself was shaded; depth (optional) is the expected depth sum(alpha T z) of the
 * blended Gaussians, the usual 3DGS depth render; rgb_alt (optional) is the colour with
 * the pixel's nearest threshold decision flipped (see or_shade); n_blend (optional) counts
 * the Gaussians blended into the shaded pixel. */
void or_render(int n, const float *rec, const int32_t *rect, const or_camera *cam, int tile,
               const uint8_t *level, const int32_t *pix, int n_pix, float *rgb,
               float *t_final, int32_t *n_contrib, int32_t *n_eval, float *margin,
               uint8_t *rendered, float *depth, float *rgb_alt, int32_t *n_blend) {
  int n_vis = 0;
  or_entry *list = or_global_list(n, rec, rect, &n_vis);
  const int W = cam->width, H = cam->height;
  const int tiles_x = or_tiles(W, tile);
  const int64_t count = pix ? (int64_t)n_pix : (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < count; ++p) {
    int x, y;
    if (pix) { x = pix[2 * p]; y = pix[2 * p + 1]; }
    else { x = (int)(p % W); y = (int)(p / W); }
    int sx = x, sy = y;
    int live = 1;
    if (level) {
      const int lv = level[(y / tile) * tiles_x + (x / tile)];
      live = or_label(x, y) <= lv;
      if (!live) { sx = x & ~1; sy = y & ~1; }
    }
    or_shade(sx, sy, tile, rec, rect, list, n_vis, rgb + 3 * p, t_final + p, n_contrib + p,
             n_eval + p, margin + p, depth ? depth + p : NULL, rgb_alt ? rgb_alt + 3 * p : NULL,
             n_blend ? n_blend + p : NULL);
    if (rendered) rendered[p] = (uint8_t)live;
  }
  free(list);
}

/* Convenience: preprocess + render of one eye in one call (used for CPU timing). */
void or_render_eye(int n, int degree, const float *means, const float *log_scales,
                   const float *quats, const float *opacity_logits, const float *sh,
                   const or_camera *cam, int tile, const or_fovea *fv, const float gaze[2],
                   const int32_t *pix, int n_pix, float *rgb, float *t_final,
                   int32_t *n_contrib, int32_t *n_eval, float *margin, uint8_t *rendered) {
  float *rec = (float *)malloc(sizeof(float) * OR_REC * (size_t)(n > 0 ? n : 1));
  int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
  uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  or_preprocess(n, degree, means, log_scales, quats, opacity_logits, sh, cam, tile, rec, rect,
                touched);
  uint8_t *level = NULL;
  if (fv) {
    const int nt = or_tiles(cam->width, tile) * or_tiles(cam->height, tile);
    level = (uint8_t *)malloc((size_t)nt);
    or_level_map(cam, tile, fv, gaze, level);
  }
  or_render(n, rec, rect, cam, tile, level, pix, n_pix, rgb, t_final, n_contrib, n_eval,
            margin, rendered, NULL, NULL, NULL);
  free(level);
  free(touched);
  free(rect);
  free(rec);
}

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
