/*
 * mlps_oracle.c -- plain FP64 CPU oracle for MLP-Splatting rendering.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package's smoke check and the benchmark's
 * CPU-baseline leg may load this library. The CUDA library never includes, links or calls it,
 * and it shares no header, helper or constant with the CUDA sources.
 *
 * What it computes, step by step, per pixel and in FP64 from the (FP32-representable) inputs:
 *
 *  1. Camera ray r(t) = o + t d with unit d through the pixel centre (Sec. 3.2).
 *  2. For EVERY primitive (brute force, no tile binning): the unit-Mahalanobis ellipsoid of
 *     centre mu, scales s and rotation R(q/|q|) (Sec. 3.1). In the primitive's scale-normalised
 *     frame o' = S^-1 R^T (o - mu), d' = S^-1 R^T d. The soft contact point of Eq. 2 is
 *     t_mid = d^T Lambda (mu - o) / d^T Lambda d = -(o'.d') / (d'.d'), Lambda = R S^-2 R^T
 *     (Eq. 1-2). The ray hits iff the squared normalised distance m2 = |o' + t_mid d'|^2 < 1.
 *     Then the chord is [t_mid - h, t_mid + h], h = sqrt((1 - m2) / (d'.d')); t_mid is its
 *     midpoint. The interval is clipped below at the camera's near distance.
 *  3. Hits are ordered by the sort key max(0, t_mid) of Eq. 2 (Sec. 3.3: per-pixel exact
 *     order), ties broken by (t0, primitive index).
 *  4. S midpoint samples per hit interval, t_k = t0 + (k + 1/2) Delta, Delta = (t1 - t0) / S;
 *     the sample's local position is x'_k = o' + t_k d'.
 *  5. Input encoding gamma of Eq. 5, per scalar sin/cos(2^l pi p) for l < L, interleaved by
 *     frequency, no identity term, concatenated component by component: local xyz first, then
 *     the world view direction d. L = 0 for xyz means the raw 3-vector; L = 0 for the
 *     direction means no direction input.
 *  6. The primitive's own MLP (Sec. 3.1): ReLU hidden layers, linear last layer.
 *  7. Output activations of Sec. 3.2: c = sigmoid, sigma = softplus; extra outputs (features)
 *     are linear.
 *  8. Front-to-back compositing of Eq. 6 over all samples in order,
 *     C = sum_j T_j alpha_j c_j, alpha_j = 1 - exp(-sigma_j Delta_j),
 *     T_j = exp(-sum_{l<j} sigma_l Delta_l), with no early termination; black background;
 *     T_final is returned. Features are composited with the same weights (Sec. 3.4).
 *  9. Reverse mode of steps 2-8 written by hand (the gradient of a scalar loss L given
 *     dL/dC, dL/dT_final and dL/dF). Hit sets and orders are piecewise constant and are not
 *     differentiated.
 *
 * Contact-point mode (contact = 1, the paper's own formulation of Sec. 3.2): one sample per hit
 * (S = 1), whose MLP input is not the sample position but the 6-vector x = [d; delta] of Eq. 4:
 * the unit view direction d and the residual delta = mu - p* from the soft contact point
 * p* = o + t* d, t* = max(0, d^T Lambda (mu - o) / d^T Lambda d) (Eq. 2-3), each component
 * encoded by gamma (L = dir_freqs for d, xyz_freqs for delta; 0 = raw). The alpha of the hit is
 * still 1 - exp(-sigma * chord length).
 *
 * Feature slots (slot_dim = C > 0, Sec. 3.4): every primitive also carries four slot embeddings
 * e_k in R^C, stored after its MLP parameters. A hit's slot feature is f = sum_k g_k e_k with
 * g = softmax_k(a_k . u), u = clip_[-1,1]^3(R^T delta / s) the scale-normalised offset of the
 * centre from the contact point (delta = mu - p* as above) and a_k the unit vertices of a
 * regular tetrahedron. The rendered slot feature map is F_slot = sum_i w_i f_i with w_i the
 * hit's compositing weight (the sum of T alpha over its samples; T_i alpha_i for S = 1). It is
 * returned after the MLP's extra outputs.
 *
 * Tile-centre ordering (tile_sort = T > 0, Sec. 3.3 and App. A.4): the image is cut into T x T
 * tiles, and every pixel composites its hits in the order of the sort key max(0, t*) computed
 * for the virtual ray through its tile's centre (image point (T tx + T/2, T ty + T/2)) instead
 * of its own ray, ties by primitive index. Hit sets, intervals, samples and MLP inputs stay the
 * pixel's own.
 *
 * Readings of points the paper leaves open (scalar delta of Eq. 6 = the sample step, support
 * = unit-Mahalanobis ellipsoid, falloff off, interval-by-interval compositing, tie-break,
 * camera model, background) are listed with the design notes of the repository.
 *
 * Threads: pixels are split over pthreads; each pixel is computed independently.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_MAX_LAYERS 16

typedef struct {
  int xyz_freqs;     /* L of gamma for the local position; 0 = raw 3-vector */
  int dir_freqs;     /* L of gamma for the view direction; 0 = no direction input */
  int hidden_width;
  int hidden_layers;
  int feat_dim;      /* extra linear outputs, composited like colour */
  int samples;       /* S midpoint samples per hit interval */
  int contact;       /* 1: contact-point mode (S = 1, input gamma([d; delta])) */
  int slot_dim;      /* C of the four slot embeddings per primitive (Sec. 3.4); 0 = none */
  int tile_sort;     /* T > 0: order hits by the tile-centre virtual ray of T x T tiles; 0 = exact */
} orc_cfg;

typedef struct {
  int width, height;
  double fx, fy, cx, cy;
  double w2c[12];    /* row-major [R | t], world -> camera, OpenCV axes */
  double near_t;
} orc_cam;

/* ------------------------------------------------------------------------------------------ */
/* Model shape                                                                                  */

int orc_input_dim(const orc_cfg* c) {
  int nx = c->xyz_freqs > 0 ? 6 * c->xyz_freqs : 3;
  int nd = c->dir_freqs > 0 ? 6 * c->dir_freqs : 0;
  return nx + nd;
}

int orc_output_dim(const orc_cfg* c) { return 4 + c->feat_dim; }

int orc_num_layers(const orc_cfg* c) { return c->hidden_layers + 1; }

static void layer_dims(const orc_cfg* c, int l, int* in, int* out) {
  int L = orc_num_layers(c);
  *in = (l == 0) ? orc_input_dim(c) : c->hidden_width;
  *out = (l == L - 1) ? orc_output_dim(c) : c->hidden_width;
}

long orc_param_count(const orc_cfg* c) {
  long n = 0;
  for (int l = 0; l < orc_num_layers(c); ++l) {
    int fi, fo;
    layer_dims(c, l, &fi, &fo);
    n += (long)fi * fo + fo;
  }
  return n + 4L * c->slot_dim;
}

static int cfg_valid(const orc_cfg* c) {
  if (c->xyz_freqs < 0 || c->dir_freqs < 0 || c->hidden_width <= 0 || c->hidden_layers < 0 ||
      c->feat_dim < 0 || c->samples <= 0)
    return 0;
  if (c->contact != 0 && (c->contact != 1 || c->samples != 1)) return 0;
  if (c->slot_dim < 0 || c->tile_sort < 0) return 0;
  if (orc_num_layers(c) > ORC_MAX_LAYERS) return 0;
  return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry                                                                                     */

typedef struct {
  double mu[3], s[3];
  double q[4];       /* as given (w, x, y, z) */
  double qn[4];      /* normalised */
  double qlen;
  double R[9];       /* R(qn), row-major */
  double M[9];       /* S^-1 R^T, row-major: maps world offsets to the normalised frame */
} prim_geo;

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void prim_setup(const double* mu, const double* s, const double* q, prim_geo* g) {
  for (int i = 0; i < 3; ++i) { g->mu[i] = mu[i]; g->s[i] = s[i]; }
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  g->qlen = n;
  for (int i = 0; i < 4; ++i) { g->q[i] = q[i]; g->qn[i] = q[i] / n; }
  quat_to_rot(g->qn, g->R);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g->M[i * 3 + j] = g->R[j * 3 + i] / s[i];
}

/* Ray through the image point (u, v) (pixel x covers [x, x + 1); its centre is x + 1/2). */
static void make_ray_uv(const orc_cam* cam, double u, double v, double* o, double* d) {
  const double* P = cam->w2c;
  double dc[3] = {(u - cam->cx) / cam->fx, (v - cam->cy) / cam->fy, 1.0};
  double t[3] = {P[3], P[7], P[11]};
  for (int i = 0; i < 3; ++i) {
    /* R^T: column i of R = (P[i], P[4+i], P[8+i]) */
    o[i] = -(P[i] * t[0] + P[4 + i] * t[1] + P[8 + i] * t[2]);
    d[i] = P[i] * dc[0] + P[4 + i] * dc[1] + P[8 + i] * dc[2];
  }
  double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int i = 0; i < 3; ++i) d[i] /= n;
}

static void make_ray(const orc_cam* cam, int x, int y, double* o, double* d) {
  make_ray_uv(cam, x + 0.5, y + 0.5, o, d);
}

typedef struct {
  int prim;
  int clamped;        /* t0 was clipped at the near distance */
  double key;         /* max(0, t_mid), Eq. 2 */
  double tmid, h, t0, t1, m2;
  double op[3], dp[3];
} hit_t;

static void matvec3(const double* M, const double* v, double* r) {
  for (int i = 0; i < 3; ++i) r[i] = M[i * 3] * v[0] + M[i * 3 + 1] * v[1] + M[i * 3 + 2] * v[2];
}

/* Returns 1 and fills *hit when the ray meets the primitive's ellipsoid in front of near. The
 * squared normalised distance m2 is always written (it decides the hit). */
static int intersect(const prim_geo* g, const double* o, const double* d, double near_t, int prim,
                     hit_t* hit, double* m2_out) {
  double rel[3] = {o[0] - g->mu[0], o[1] - g->mu[1], o[2] - g->mu[2]};
  double op[3], dp[3];
  matvec3(g->M, rel, op);
  matvec3(g->M, d, dp);
  double a = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  double b = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
  double tmid = -b / a;
  double p[3] = {op[0] + tmid * dp[0], op[1] + tmid * dp[1], op[2] + tmid * dp[2]};
  double m2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  if (m2_out) *m2_out = m2;
  if (!(m2 < 1.0)) return 0;
  double h = sqrt((1.0 - m2) / a);
  double t0 = tmid - h, t1 = tmid + h;
  int clamped = 0;
  if (t0 < near_t) { t0 = near_t; clamped = 1; }
  if (!(t1 > t0)) return 0;
  hit->prim = prim;
  hit->clamped = clamped;
  hit->tmid = tmid;
  hit->key = tmid > 0 ? tmid : 0;
  hit->h = h;
  hit->t0 = t0;
  hit->t1 = t1;
  hit->m2 = m2;
  for (int i = 0; i < 3; ++i) { hit->op[i] = op[i]; hit->dp[i] = dp[i]; }
  return 1;
}

static int hit_cmp(const void* pa, const void* pb) {
  const hit_t* a = (const hit_t*)pa;
  const hit_t* b = (const hit_t*)pb;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  if (a->t0 < b->t0) return -1;
  if (a->t0 > b->t0) return 1;
  return (a->prim > b->prim) - (a->prim < b->prim);
}

static int hit_cmp_tile(const void* pa, const void* pb) {
  const hit_t* a = (const hit_t*)pa;
  const hit_t* b = (const hit_t*)pb;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  return (a->prim > b->prim) - (a->prim < b->prim);
}

/* Order a pixel's hits: by its own max(0, t*) (Eq. 2), or with tile > 0 by max(0, t*) of the
 * virtual ray through the centre of the pixel's tile, d^T Lambda (mu - o) / d^T Lambda d with
 * that ray's d (Sec. 3.3). The hits keep their own intervals; only key and order change. */
static void order_hits(const prim_geo* geo, const orc_cam* cam, int x, int y, int tile, hit_t* hits, int nh) {
  if (tile <= 0) {
    qsort(hits, (size_t)nh, sizeof(hit_t), hit_cmp);
    return;
  }
  double oc[3], dc[3];
  make_ray_uv(cam, (double)(x / tile) * tile + 0.5 * tile, (double)(y / tile) * tile + 0.5 * tile, oc, dc);
  for (int i = 0; i < nh; ++i) {
    const prim_geo* g = &geo[hits[i].prim];
    double op[3], dp[3];
    for (int r = 0; r < 3; ++r) {
      op[r] = 0; dp[r] = 0;
      for (int cc = 0; cc < 3; ++cc) {
        op[r] += g->M[r * 3 + cc] * (oc[cc] - g->mu[cc]);
        dp[r] += g->M[r * 3 + cc] * dc[cc];
      }
    }
    double ts = -(op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2]) / (dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
    hits[i].key = ts > 0 ? ts : 0;
  }
  qsort(hits, (size_t)nh, sizeof(hit_t), hit_cmp_tile);
}

/* ------------------------------------------------------------------------------------------ */
/* Encoding and MLP                                                                             */

static int encode(const orc_cfg* c, const double* xl, const double* d, double* e) {
  int n = 0;
  if (c->xyz_freqs == 0) {
    for (int i = 0; i < 3; ++i) e[n++] = xl[i];
  } else {
    for (int i = 0; i < 3; ++i)
      for (int l = 0; l < c->xyz_freqs; ++l) {
        double f = ldexp(M_PI, l) * xl[i];
        e[n++] = sin(f);
        e[n++] = cos(f);
      }
  }
  if (c->dir_freqs > 0) {
    for (int i = 0; i < 3; ++i)
      for (int l = 0; l < c->dir_freqs; ++l) {
        double f = ldexp(M_PI, l) * d[i];
        e[n++] = sin(f);
        e[n++] = cos(f);
      }
  }
  return n;
}

/* d gamma / d xl chained: given the gradient on the encoding, add dL/dxl. */
static void encode_backward(const orc_cfg* c, const double* xl, const double* ge, double* gx) {
  if (c->xyz_freqs == 0) {
    for (int i = 0; i < 3; ++i) gx[i] += ge[i];
    return;
  }
  int n = 0;
  for (int i = 0; i < 3; ++i)
    for (int l = 0; l < c->xyz_freqs; ++l) {
      double w = ldexp(M_PI, l);
      double f = w * xl[i];
      gx[i] += ge[n] * w * cos(f) - ge[n + 1] * w * sin(f);
      n += 2;
    }
}

/* gamma of one 3-vector with L frequencies (raw when L = 0), appended at e[n]. */
static int encode_vec(int L, const double* v, double* e, int n) {
  if (L == 0) {
    for (int i = 0; i < 3; ++i) e[n++] = v[i];
    return n;
  }
  for (int i = 0; i < 3; ++i)
    for (int l = 0; l < L; ++l) {
      double f = ldexp(M_PI, l) * v[i];
      e[n++] = sin(f);
      e[n++] = cos(f);
    }
  return n;
}

/* Contact-point mode input gamma([d; delta]) (Eq. 4-5): direction first, then the residual. */
static int encode_contact(const orc_cfg* c, const double* d, const double* delta, double* e) {
  int n = 0;
  if (c->dir_freqs > 0) n = encode_vec(c->dir_freqs, d, e, n);
  return encode_vec(c->xyz_freqs, delta, e, n);
}

/* dL/d delta from the gradient on the contact-mode encoding. */
static void encode_contact_backward(const orc_cfg* c, const double* delta, const double* ge, double* gdelta) {
  int n = c->dir_freqs > 0 ? 6 * c->dir_freqs : 0;
  if (c->xyz_freqs == 0) {
    for (int i = 0; i < 3; ++i) gdelta[i] = ge[n + i];
    return;
  }
  for (int i = 0; i < 3; ++i) {
    gdelta[i] = 0;
    for (int l = 0; l < c->xyz_freqs; ++l) {
      double w = ldexp(M_PI, l);
      double f = w * delta[i];
      gdelta[i] += ge[n] * w * cos(f) - ge[n + 1] * w * sin(f);
      n += 2;
    }
  }
}

/* delta = mu - p*, p* = o + t* d, t* = max(0, t_mid) (Eq. 2-3). */
static void contact_delta(const double* mu, const double* o, const double* d, double tmid, double* delta) {
  double ts = tmid > 0 ? tmid : 0;
  for (int i = 0; i < 3; ++i) delta[i] = mu[i] - (o[i] + ts * d[i]);
}

typedef struct {
  const orc_cfg* cfg;
  int nl, nin, nout, width;
  long P;        /* MLP parameters per primitive */
  long Prow;     /* all parameters per primitive: the MLP's, then 4 slot embeddings of C */
  int C;         /* slot dimension */
  long woff[ORC_MAX_LAYERS], boff[ORC_MAX_LAYERS];
  int din[ORC_MAX_LAYERS], dout[ORC_MAX_LAYERS];
  long act_size; /* doubles for all layer inputs + the final output */
} model_t;

static void model_init(model_t* m, const orc_cfg* c) {
  m->cfg = c;
  m->nl = orc_num_layers(c);
  m->nin = orc_input_dim(c);
  m->nout = orc_output_dim(c);
  m->width = c->hidden_width;
  long off = 0, act = 0;
  for (int l = 0; l < m->nl; ++l) {
    layer_dims(c, l, &m->din[l], &m->dout[l]);
    m->woff[l] = off;
    off += (long)m->din[l] * m->dout[l];
    m->boff[l] = off;
    off += m->dout[l];
    act += m->din[l];
  }
  m->P = off;
  m->C = c->slot_dim;
  m->Prow = off + 4L * c->slot_dim;
  m->act_size = act + m->nout;
}

/* acts holds the input of every layer in order, then the raw last-layer output. */
static void mlp_forward(const model_t* m, const double* w, double* acts) {
  double* in = acts;
  for (int l = 0; l < m->nl; ++l) {
    double* out = in + m->din[l];
    const double* W = w + m->woff[l];
    const double* b = w + m->boff[l];
    for (int j = 0; j < m->dout[l]; ++j) {
      double acc = b[j];
      for (int k = 0; k < m->din[l]; ++k) acc += W[(long)j * m->din[l] + k] * in[k];
      if (l < m->nl - 1 && acc < 0) acc = 0; /* ReLU on hidden layers */
      out[j] = acc;
    }
    in = out;
  }
}

/* Backward of mlp_forward: gout = dL/d(raw output); adds into gw; writes dL/d(input) to gin. */
static void mlp_backward(const model_t* m, const double* w, const double* acts, const double* gout,
                         double* gw, double* gin, double* buf_a, double* buf_b) {
  /* offsets of each layer's input within acts */
  long aoff[ORC_MAX_LAYERS + 1];
  aoff[0] = 0;
  for (int l = 0; l < m->nl; ++l) aoff[l + 1] = aoff[l] + m->din[l];
  double* delta = buf_a;
  double* next = buf_b;
  for (int j = 0; j < m->nout; ++j) delta[j] = gout[j];
  for (int l = m->nl - 1; l >= 0; --l) {
    const double* in = acts + aoff[l];
    const double* W = w + m->woff[l];
    double* gW = gw + m->woff[l];
    double* gb = gw + m->boff[l];
    int fi = m->din[l], fo = m->dout[l];
    for (int j = 0; j < fo; ++j) {
      gb[j] += delta[j];
      for (int k = 0; k < fi; ++k) gW[(long)j * fi + k] += delta[j] * in[k];
    }
    for (int k = 0; k < fi; ++k) {
      double acc = 0;
      for (int j = 0; j < fo; ++j) acc += W[(long)j * fi + k] * delta[j];
      /* the input of layer l > 0 is a ReLU output of layer l-1 */
      if (l > 0 && !(in[k] > 0)) acc = 0;
      next[k] = acc;
    }
    double* t = delta; delta = next; next = t;
  }
  for (int k = 0; k < m->nin; ++k) gin[k] = delta[k];
}

static double sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }
static double softplus(double z) { return (z > 0 ? z : 0) + log1p(exp(-fabs(z))); }

/* ------------------------------------------------------------------------------------------ */
/* Per-pixel render (+ optional reverse mode)                                                   */

/* ------------------------------------------------------------------------------------------ */
/* Feature slots (Sec. 3.4)                                                                     */

/* The four directions a_k: unit vertices of a regular tetrahedron, (+-1, +-1, +-1)/sqrt(3) with
 * an even number of minus signs. */
static void slot_frame(double a[4][3]) {
  const double v[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) a[k][c] = v[k][c] / sqrt(3.0);
}

/* g = softmax_k(a_k . u) */
static void slot_softmax(const double* u, double* g) {
  double a[4][3], z[4], zmax = -1e300, sum = 0;
  slot_frame(a);
  for (int k = 0; k < 4; ++k) {
    z[k] = a[k][0] * u[0] + a[k][1] * u[1] + a[k][2] * u[2];
    if (z[k] > zmax) zmax = z[k];
  }
  for (int k = 0; k < 4; ++k) { g[k] = exp(z[k] - zmax); sum += g[k]; }
  for (int k = 0; k < 4; ++k) g[k] /= sum;
}

/* y = M delta (M = S^-1 R^T), u = clip(y) to [-1, 1]^3 */
static void slot_offset(const double* M, const double* delta, double* y, double* u) {
  for (int r = 0; r < 3; ++r) {
    y[r] = M[r * 3] * delta[0] + M[r * 3 + 1] * delta[1] + M[r * 3 + 2] * delta[2];
    u[r] = y[r] < -1 ? -1 : (y[r] > 1 ? 1 : y[r]);
  }
}

typedef struct {
  const orc_cfg* cfg;
  model_t model;
  int K;
  prim_geo* geo;
  const double* weights; /* [K, P] */
  int n_views;
  const orc_cam* cams;
  int n_pix;
  const int* pix;        /* [n_pix, 3] (view, x, y) */
  double *rgb, *trans, *feat; /* per listed pixel */
  /* backward */
  const double *g_rgb, *g_trans, *g_feat;
  double *d_weights, *d_centers, *d_scales, *d_quats; /* d_* of M and mu first, then chained */
  double* d_M;           /* [K, 9] accumulated dL/dM */
  double* d_mu;          /* [K, 3] */
  pthread_mutex_t* locks;/* one per primitive */
  int status;
} job_t;

typedef struct {
  job_t* job;
  int begin, end;
  int status;
} slice_t;

typedef struct {
  hit_t* hits;
  double* samp;     /* per sample: [nout activated outputs, a = sigma*Delta, T before] */
  double* acts;
  double* enc_g;
  double* gw;       /* per-hit weight gradient scratch [P] */
  double *buf_a, *buf_b;
  double* gout;
  long samp_cap;
} scratch_t;

static int scratch_init(scratch_t* s, const job_t* j) {
  const model_t* m = &j->model;
  int maxw = m->nin;
  for (int l = 0; l < m->nl; ++l) if (m->dout[l] > maxw) maxw = m->dout[l];
  s->hits = (hit_t*)malloc(sizeof(hit_t) * (size_t)(j->K > 0 ? j->K : 1));
  s->acts = (double*)malloc(sizeof(double) * (size_t)m->act_size);
  s->enc_g = (double*)malloc(sizeof(double) * (size_t)m->nin);
  s->gw = j->d_weights ? (double*)calloc((size_t)m->Prow, sizeof(double)) : NULL;
  s->buf_a = (double*)malloc(sizeof(double) * (size_t)maxw);
  s->buf_b = (double*)malloc(sizeof(double) * (size_t)maxw);
  s->gout = (double*)malloc(sizeof(double) * (size_t)m->nout);
  s->samp = NULL;
  s->samp_cap = 0;
  return s->hits && s->acts && s->enc_g && s->buf_a && s->buf_b && s->gout &&
         (!j->d_weights || s->gw);
}

static void scratch_free(scratch_t* s) {
  free(s->hits); free(s->acts); free(s->enc_g); free(s->gw);
  free(s->buf_a); free(s->buf_b); free(s->gout); free(s->samp);
}

/* Evaluate sample k of a hit: encodes, runs the MLP into s->acts, returns x' in xl (contact
 * mode: the residual delta of Eq. 3 in xl). */
static void eval_sample(const job_t* j, const hit_t* h, const double* o, const double* d, int k,
                        scratch_t* s, double* xl, double* tk_out) {
  int S = j->cfg->samples;
  double delta = (h->t1 - h->t0) / S;
  double tk = h->t0 + (k + 0.5) * delta;
  if (j->cfg->contact) {
    contact_delta(j->geo[h->prim].mu, o, d, h->tmid, xl);
    encode_contact(j->cfg, d, xl, s->acts);
  } else {
    for (int i = 0; i < 3; ++i) xl[i] = h->op[i] + tk * h->dp[i];
    encode(j->cfg, xl, d, s->acts);
  }
  mlp_forward(&j->model, j->weights + (long)h->prim * j->model.Prow, s->acts);
  if (tk_out) *tk_out = tk;
}

static int render_pixel(job_t* j, int idx, scratch_t* s) {
  const orc_cfg* c = j->cfg;
  const model_t* m = &j->model;
  int v = j->pix[3 * idx], x = j->pix[3 * idx + 1], y = j->pix[3 * idx + 2];
  const orc_cam* cam = &j->cams[v];
  double o[3], d[3];
  make_ray(cam, x, y, o, d);
  int nh = 0;
  for (int p = 0; p < j->K; ++p)
    if (intersect(&j->geo[p], o, d, cam->near_t, p, &s->hits[nh], NULL)) ++nh;
  order_hits(j->geo, cam, x, y, c->tile_sort, s->hits, nh);

  int S = c->samples, F = c->feat_dim, NO = m->nout;
  long ns = (long)nh * S;
  long rec = NO + 2;
  if (ns * rec > s->samp_cap) {
    free(s->samp);
    s->samp_cap = ns * rec;
    s->samp = (double*)malloc(sizeof(double) * (size_t)s->samp_cap);
    if (!s->samp) return 1;
  }
  const double* out = s->acts + (m->act_size - NO);
  const int Cs = m->C, FT = F + Cs; /* feature row: the MLP's F outputs, then the C slot channels */
  double C[3] = {0, 0, 0};
  double* Fo = j->feat ? j->feat + (long)idx * FT : NULL;
  if (Fo) for (int f = 0; f < FT; ++f) Fo[f] = 0;
  double A = 0; /* accumulated optical depth: T = exp(-A) */
  double xl[3];
  for (int hi = 0; hi < nh; ++hi) {
    const hit_t* h = &s->hits[hi];
    double delta = (h->t1 - h->t0) / S;
    double wh = 0; /* the hit's compositing weight */
    for (int k = 0; k < S; ++k) {
      eval_sample(j, h, o, d, k, s, xl, NULL);
      double* r = s->samp + ((long)hi * S + k) * rec;
      r[0] = sigmoid(out[0]); r[1] = sigmoid(out[1]); r[2] = sigmoid(out[2]);
      r[3] = softplus(out[3]);
      for (int f = 0; f < F; ++f) r[4 + f] = out[4 + f];
      double a = r[3] * delta;
      double T = exp(-A);
      double alpha = 1.0 - exp(-a);
      r[NO] = a;
      r[NO + 1] = T;
      for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * r[ch];
      if (Fo) for (int f = 0; f < F; ++f) Fo[f] += T * alpha * r[4 + f];
      wh += T * alpha;
      A += a;
    }
    if (Fo && Cs > 0) {
      /* F_slot += w_i sum_k g_k e_k (Sec. 3.4) */
      double dl[3], yv[3], u[3], g[4];
      contact_delta(j->geo[h->prim].mu, o, d, h->tmid, dl);
      slot_offset(j->geo[h->prim].M, dl, yv, u);
      slot_softmax(u, g);
      const double* e = j->weights + (long)h->prim * m->Prow + m->P;
      for (int ch = 0; ch < Cs; ++ch)
        Fo[F + ch] += wh * (g[0] * e[ch] + g[1] * e[Cs + ch] + g[2] * e[2 * Cs + ch] + g[3] * e[3 * Cs + ch]);
    }
  }
  double Tfin = exp(-A);
  if (j->rgb) for (int ch = 0; ch < 3; ++ch) j->rgb[(long)idx * 3 + ch] = C[ch];
  if (j->trans) j->trans[idx] = Tfin;
  if (!j->d_weights) return 0;

  /* ---- reverse mode ---- */
  double gC[3] = {0, 0, 0}, gT = 0;
  if (j->g_rgb) for (int ch = 0; ch < 3; ++ch) gC[ch] = j->g_rgb[(long)idx * 3 + ch];
  if (j->g_trans) gT = j->g_trans[idx];
  const double* gF = (j->g_feat && F > 0) ? j->g_feat + (long)idx * FT : NULL;
  const double* gFs = (j->g_feat && Cs > 0) ? j->g_feat + (long)idx * FT + F : NULL;
  double Rs = 0; /* sum over later samples of T alpha (f . dL/dF_slot) */
  double Rrgb[3] = {0, 0, 0};   /* sum over later samples of T alpha c */
  double RF[64];
  if (F > 64) return 2;
  for (int f = 0; f < F; ++f) RF[f] = 0;
  for (int hi = nh - 1; hi >= 0; --hi) {
    const hit_t* h = &s->hits[hi];
    int P = h->prim;
    double delta = (h->t1 - h->t0) / S;
    memset(s->gw, 0, sizeof(double) * (size_t)m->Prow);
    double g_op[3] = {0, 0, 0}, g_dp[3] = {0, 0, 0}, g_t0 = 0, g_t1 = 0, g_delta = 0;
    double g_mu_direct[3] = {0, 0, 0}, g_tmid_direct = 0; /* contact mode and slots */
    double g_M_direct[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};     /* slots: through u = clip(M delta) */
    /* slots: the hit's offset, slot weights and s_k = e_k . dL/dF_slot */
    double sdl[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, su[3], sg[4] = {0, 0, 0, 0}, ss[4] = {0, 0, 0, 0};
    double s_hit = 0, wh = 0;
    const double* e_slot = j->weights + (long)P * m->Prow + m->P;
    if (gFs) {
      contact_delta(j->geo[P].mu, o, d, h->tmid, sdl);
      slot_offset(j->geo[P].M, sdl, sy, su);
      slot_softmax(su, sg);
      for (int k = 0; k < 4; ++k) {
        for (int ch = 0; ch < Cs; ++ch) ss[k] += e_slot[k * Cs + ch] * gFs[ch];
        s_hit += sg[k] * ss[k];
      }
    }
    for (int k = S - 1; k >= 0; --k) {
      double* r = s->samp + ((long)hi * S + k) * rec;
      double a = r[NO], T = r[NO + 1];
      double ea = exp(-a);
      double alpha = 1.0 - ea;
      double w = T * alpha;
      double Tn = T * ea;
      /* dL/da of C = sum T alpha c, T_final = exp(-sum a) */
      double ga = -gT * Tfin;
      for (int ch = 0; ch < 3; ++ch) ga += gC[ch] * (Tn * r[ch] - Rrgb[ch]);
      if (gF) for (int f = 0; f < F; ++f) ga += gF[f] * (Tn * r[4 + f] - RF[f]);
      if (gFs) ga += Tn * s_hit - Rs; /* the slot feature is constant over the hit's samples */
      for (int ch = 0; ch < 3; ++ch) Rrgb[ch] += w * r[ch];
      if (gF) for (int f = 0; f < F; ++f) RF[f] += w * r[4 + f];
      if (gFs) Rs += w * s_hit;
      wh += w;
      double gsigma = ga * delta;
      g_delta += ga * r[3];
      /* recompute the MLP for this sample */
      double tk;
      eval_sample(j, h, o, d, k, s, xl, &tk);
      for (int ch = 0; ch < 3; ++ch) s->gout[ch] = w * gC[ch] * r[ch] * (1.0 - r[ch]);
      s->gout[3] = gsigma * sigmoid(out[3]);
      for (int f = 0; f < F; ++f) s->gout[4 + f] = gF ? w * gF[f] : 0.0;
      mlp_backward(m, j->weights + (long)P * m->Prow, s->acts, s->gout, s->gw, s->enc_g, s->buf_a,
                   s->buf_b);
      double gx[3] = {0, 0, 0};
      if (c->contact) {
        /* delta = mu - o - t* d: dL/dmu directly, and through t* = t_mid when t_mid > 0 */
        double gd[3];
        encode_contact_backward(c, xl, s->enc_g, gd);
        for (int i = 0; i < 3; ++i) g_mu_direct[i] += gd[i];
        if (h->tmid > 0) g_tmid_direct -= gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
      } else {
        encode_backward(c, xl, s->enc_g, gx);
      }
      /* x' = o' + t_k d',  t_k = t0 + (k + 1/2)(t1 - t0)/S */
      double gt = 0;
      for (int i = 0; i < 3; ++i) {
        g_op[i] += gx[i];
        g_dp[i] += tk * gx[i];
        gt += gx[i] * h->dp[i];
      }
      double u = (k + 0.5) / S;
      g_t0 += gt * (1.0 - u);
      g_t1 += gt * u;
    }
    if (gFs) {
      /* dL/de_k = w g_k dL/dF_slot; dL/dg_k = w s_k; softmax; u = clip(y), y = M delta */
      for (int k = 0; k < 4; ++k)
        for (int ch = 0; ch < Cs; ++ch) s->gw[m->P + k * Cs + ch] += wh * sg[k] * gFs[ch];
      double a4[4][3], gz[4], mean = 0, gy[3] = {0, 0, 0};
      slot_frame(a4);
      for (int k = 0; k < 4; ++k) mean += sg[k] * wh * ss[k];
      for (int k = 0; k < 4; ++k) gz[k] = sg[k] * (wh * ss[k] - mean);
      for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 4; ++k) gy[r] += gz[k] * a4[k][r];
        if (sy[r] < -1 || sy[r] > 1) gy[r] = 0;
      }
      /* y = M delta: dL/dM += gy delta^T, dL/d delta = M^T gy; delta = mu - o - max(0, t_mid) d */
      const double* Mg = j->geo[P].M;
      double gdl[3];
      for (int cc = 0; cc < 3; ++cc) {
        gdl[cc] = Mg[cc] * gy[0] + Mg[3 + cc] * gy[1] + Mg[6 + cc] * gy[2];
        for (int r = 0; r < 3; ++r) g_M_direct[r * 3 + cc] += gy[r] * sdl[cc];
        g_mu_direct[cc] += gdl[cc];
      }
      if (h->tmid > 0) g_tmid_direct -= gdl[0] * d[0] + gdl[1] * d[1] + gdl[2] * d[2];
    }
    g_t0 -= g_delta / S;
    g_t1 += g_delta / S;
    /* t0 = t_mid - h (unless clipped at near), t1 = t_mid + h */
    double g_tmid = g_t1 + (h->clamped ? 0.0 : g_t0) + g_tmid_direct;
    double g_h = g_t1 - (h->clamped ? 0.0 : g_t0);
    const double* op = h->op;
    const double* dp = h->dp;
    double a = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    double b = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
    double oo = op[0] * op[0] + op[1] * op[1] + op[2] * op[2];
    double hh = h->h;
    for (int i = 0; i < 3; ++i) {
      /* t_mid = -b/a */
      g_op[i] += g_tmid * (-dp[i] / a);
      g_dp[i] += g_tmid * (-op[i] / a + 2.0 * b * dp[i] / (a * a));
      /* h = sqrt(a (1 - |o'|^2) + b^2) / a */
      g_op[i] += g_h * ((-a * op[i] + b * dp[i]) / (a * a * hh));
      g_dp[i] += g_h * ((dp[i] * (1.0 - oo) + b * op[i]) / (a * a * hh) - 2.0 * hh * dp[i] / a);
    }
    /* o' = M (o - mu), d' = M d */
    const prim_geo* g = &j->geo[P];
    double rel[3] = {o[0] - g->mu[0], o[1] - g->mu[1], o[2] - g->mu[2]};
    double dM[9], dmu[3];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) dM[r * 3 + cc] = g_op[r] * rel[cc] + g_dp[r] * d[cc] + g_M_direct[r * 3 + cc];
    for (int cc = 0; cc < 3; ++cc)
      dmu[cc] = -(g->M[0 * 3 + cc] * g_op[0] + g->M[1 * 3 + cc] * g_op[1] + g->M[2 * 3 + cc] * g_op[2]) +
                g_mu_direct[cc];
    pthread_mutex_lock(&j->locks[P]);
    double* dW = j->d_weights + (long)P * m->Prow;
    for (long i = 0; i < m->Prow; ++i) dW[i] += s->gw[i];
    for (int i = 0; i < 9; ++i) j->d_M[P * 9 + i] += dM[i];
    for (int i = 0; i < 3; ++i) j->d_mu[P * 3 + i] += dmu[i];
    pthread_mutex_unlock(&j->locks[P]);
  }
  return 0;
}

static void* worker(void* arg) {
  slice_t* sl = (slice_t*)arg;
  scratch_t s;
  if (!scratch_init(&s, sl->job)) { scratch_free(&s); sl->status = 1; return NULL; }
  for (int i = sl->begin; i < sl->end && sl->status == 0; ++i) sl->status = render_pixel(sl->job, i, &s);
  scratch_free(&s);
  return NULL;
}

static int run_job(job_t* j, int n_threads) {
  if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > j->n_pix) n_threads = j->n_pix > 0 ? j->n_pix : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  slice_t* sl = (slice_t*)malloc(sizeof(slice_t) * (size_t)n_threads);
  if (!th || !sl) { free(th); free(sl); return 1; }
  for (int t = 0; t < n_threads; ++t) {
    sl[t].job = j;
    sl[t].begin = (int)((long)j->n_pix * t / n_threads);
    sl[t].end = (int)((long)j->n_pix * (t + 1) / n_threads);
    sl[t].status = 0;
    pthread_create(&th[t], NULL, worker, &sl[t]);
  }
  int st = 0;
  for (int t = 0; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    if (sl[t].status) st = sl[t].status;
  }
  free(th);
  free(sl);
  return st;
}

static int setup_geo(job_t* j, const double* centers, const double* scales, const double* quats) {
  j->geo = (prim_geo*)malloc(sizeof(prim_geo) * (size_t)(j->K > 0 ? j->K : 1));
  if (!j->geo) return 1;
  for (int p = 0; p < j->K; ++p) prim_setup(centers + 3 * p, scales + 3 * p, quats + 4 * p, &j->geo[p]);
  return 0;
}

static int check_pixels(const job_t* j) {
  for (int i = 0; i < j->n_pix; ++i) {
    int v = j->pix[3 * i], x = j->pix[3 * i + 1], y = j->pix[3 * i + 2];
    if (v < 0 || v >= j->n_views) return 0;
    if (x < 0 || y < 0 || x >= j->cams[v].width || y >= j->cams[v].height) return 0;
  }
  return 1;
}

/* Render the listed pixels. rgb [n_pix,3], trans [n_pix], feat [n_pix,F] (each may be NULL).
 * Returns 0 on success, nonzero on invalid input or allocation failure. */
int orc_render(const orc_cfg* cfg, int K, const double* centers, const double* scales,
               const double* quats, const double* weights, int n_views, const orc_cam* cams,
               int n_pix, const int* pix, double* rgb, double* trans, double* feat, int n_threads) {
  if (!cfg_valid(cfg) || K < 0 || n_pix < 0 || n_views <= 0) return -1;
  job_t j;
  memset(&j, 0, sizeof(j));
  j.cfg = cfg;
  model_init(&j.model, cfg);
  j.K = K; j.weights = weights; j.n_views = n_views; j.cams = cams;
  j.n_pix = n_pix; j.pix = pix; j.rgb = rgb; j.trans = trans; j.feat = feat;
  if (!check_pixels(&j)) return -1;
  if (setup_geo(&j, centers, scales, quats)) return 1;
  int st = run_job(&j, n_threads);
  free(j.geo);
  return st;
}

/* Chain dL/dM and dL/dmu (accumulated per primitive) to scales and quaternions. */
static void chain_pose(const prim_geo* g, const double* dM, const double* dmu, double* dc,
                       double* ds, double* dq) {
  for (int i = 0; i < 3; ++i) dc[i] += dmu[i];
  /* M_ij = R_ji / s_i */
  double dR[9] = {0};
  for (int i = 0; i < 3; ++i) {
    double acc = 0;
    for (int jx = 0; jx < 3; ++jx) {
      acc += dM[i * 3 + jx] * (-g->R[jx * 3 + i] / (g->s[i] * g->s[i]));
      dR[jx * 3 + i] += dM[i * 3 + jx] / g->s[i];
    }
    ds[i] += acc;
  }
  double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
  double gq[4];
  gq[0] = -2 * z * dR[1] + 2 * y * dR[2] + 2 * z * dR[3] - 2 * x * dR[5] - 2 * y * dR[6] + 2 * x * dR[7];
  gq[1] = 2 * y * dR[1] + 2 * z * dR[2] + 2 * y * dR[3] - 4 * x * dR[4] - 2 * w * dR[5] + 2 * z * dR[6] +
          2 * w * dR[7] - 4 * x * dR[8];
  gq[2] = -4 * y * dR[0] + 2 * x * dR[1] + 2 * w * dR[2] + 2 * x * dR[3] + 2 * z * dR[5] - 2 * w * dR[6] +
          2 * z * dR[7] - 4 * y * dR[8];
  gq[3] = -4 * z * dR[0] - 2 * w * dR[1] + 2 * x * dR[2] + 2 * w * dR[3] - 4 * z * dR[4] + 2 * y * dR[5] +
          2 * x * dR[6] + 2 * y * dR[7];
  /* q_n = q / |q| */
  double dot = gq[0] * g->qn[0] + gq[1] * g->qn[1] + gq[2] * g->qn[2] + gq[3] * g->qn[3];
  for (int i = 0; i < 4; ++i) dq[i] += (gq[i] - g->qn[i] * dot) / g->qlen;
}

/* Gradient of L over the listed pixels. g_rgb [n_pix,3], g_trans [n_pix] and g_feat [n_pix,F]
 * may be NULL (zero). Outputs are overwritten: d_weights [K,P], d_centers/d_scales [K,3],
 * d_quats [K,4]. rgb/trans/feat (forward results) may be NULL. */
int orc_render_backward(const orc_cfg* cfg, int K, const double* centers, const double* scales,
                        const double* quats, const double* weights, int n_views,
                        const orc_cam* cams, int n_pix, const int* pix, const double* g_rgb,
                        const double* g_trans, const double* g_feat, double* rgb, double* trans,
                        double* feat, double* d_weights, double* d_centers, double* d_scales,
                        double* d_quats, int n_threads) {
  if (!cfg_valid(cfg) || K < 0 || n_pix < 0 || n_views <= 0 || !d_weights || !d_centers ||
      !d_scales || !d_quats)
    return -1;
  if (cfg->feat_dim > 64) return -1;
  job_t j;
  memset(&j, 0, sizeof(j));
  j.cfg = cfg;
  model_init(&j.model, cfg);
  j.K = K; j.weights = weights; j.n_views = n_views; j.cams = cams;
  j.n_pix = n_pix; j.pix = pix; j.rgb = rgb; j.trans = trans; j.feat = feat;
  j.g_rgb = g_rgb; j.g_trans = g_trans; j.g_feat = g_feat;
  if (!check_pixels(&j)) return -1;
  memset(d_weights, 0, sizeof(double) * (size_t)K * (size_t)j.model.Prow);
  memset(d_centers, 0, sizeof(double) * (size_t)K * 3);
  memset(d_scales, 0, sizeof(double) * (size_t)K * 3);
  memset(d_quats, 0, sizeof(double) * (size_t)K * 4);
  j.d_weights = d_weights;
  j.d_M = (double*)calloc((size_t)(K > 0 ? K : 1) * 9, sizeof(double));
  j.d_mu = (double*)calloc((size_t)(K > 0 ? K : 1) * 3, sizeof(double));
  j.locks = (pthread_mutex_t*)malloc(sizeof(pthread_mutex_t) * (size_t)(K > 0 ? K : 1));
  if (!j.d_M || !j.d_mu || !j.locks || setup_geo(&j, centers, scales, quats)) {
    free(j.d_M); free(j.d_mu); free(j.locks);
    return 1;
  }
  for (int p = 0; p < K; ++p) pthread_mutex_init(&j.locks[p], NULL);
  int st = run_job(&j, n_threads);
  for (int p = 0; p < K; ++p) {
    chain_pose(&j.geo[p], j.d_M + 9 * p, j.d_mu + 3 * p, d_centers + 3 * p, d_scales + 3 * p,
               d_quats + 4 * p);
    pthread_mutex_destroy(&j.locks[p]);
  }
  free(j.geo); free(j.d_M); free(j.d_mu); free(j.locks);
  return st;
}

/* Sorted hit list of one pixel (tile > 0: in the tile-centre order of T x T tiles, `key` the
 * tile key): up to max_out entries of (prim, key, t0, t1, m2). Returns the number of hits (may
 * exceed max_out; only max_out are written), or -1 on invalid input. */
int orc_ray_hits(int K, const double* centers, const double* scales, const double* quats,
                 const orc_cam* cam, int x, int y, int tile, int max_out, int* prim, double* key,
                 double* t0, double* t1, double* m2) {
  if (K < 0 || tile < 0 || x < 0 || y < 0 || x >= cam->width || y >= cam->height) return -1;
  hit_t* hits = (hit_t*)malloc(sizeof(hit_t) * (size_t)(K > 0 ? K : 1));
  prim_geo* geo = (prim_geo*)malloc(sizeof(prim_geo) * (size_t)(K > 0 ? K : 1));
  if (!hits || !geo) { free(hits); free(geo); return -1; }
  double o[3], d[3];
  make_ray(cam, x, y, o, d);
  int nh = 0;
  for (int p = 0; p < K; ++p) {
    prim_setup(centers + 3 * p, scales + 3 * p, quats + 4 * p, &geo[p]);
    if (intersect(&geo[p], o, d, cam->near_t, p, &hits[nh], NULL)) ++nh;
  }
  order_hits(geo, cam, x, y, tile, hits, nh);
  free(geo);
  for (int i = 0; i < nh && i < max_out; ++i) {
    prim[i] = hits[i].prim; key[i] = hits[i].key; t0[i] = hits[i].t0; t1[i] = hits[i].t1;
    m2[i] = hits[i].m2;
  }
  free(hits);
  return nh;
}

/* Squared normalised distance m2 of one pixel's ray to every primitive (for tangency checks)
 * and the unclipped chord midpoint t_mid. */
int orc_ray_m2(int K, const double* centers, const double* scales, const double* quats,
               const orc_cam* cam, int x, int y, double* m2, double* tmid) {
  if (K < 0 || x < 0 || y < 0 || x >= cam->width || y >= cam->height) return -1;
  double o[3], d[3];
  make_ray(cam, x, y, o, d);
  for (int p = 0; p < K; ++p) {
    prim_geo g;
    hit_t h;
    prim_setup(centers + 3 * p, scales + 3 * p, quats + 4 * p, &g);
    double m;
    intersect(&g, o, d, cam->near_t, p, &h, &m);
    m2[p] = m;
    if (tmid) {
      double rel[3] = {o[0] - g.mu[0], o[1] - g.mu[1], o[2] - g.mu[2]}, op[3], dp[3];
      matvec3(g.M, rel, op);
      matvec3(g.M, d, dp);
      tmid[p] = -(op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2]) /
                (dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
    }
  }
  return 0;
}

/* Ray of one pixel (origin, unit direction), for tests. */
int orc_pixel_ray(const orc_cam* cam, int x, int y, double* o, double* d) {
  make_ray(cam, x, y, o, d);
  return 0;
}

/* Encoding of one (local position, direction) pair, for tests; in contact-point mode xl is the
 * residual delta and the result is gamma([d; delta]). Returns its length. */
int orc_encode(const orc_cfg* cfg, const double* xl, const double* d, double* out) {
  if (cfg->contact) return encode_contact(cfg, d, xl, out);
  return encode(cfg, xl, d, out);
}

/* Slot weights g = softmax_k(a_k . u) of an offset u (Sec. 3.4), for tests. */
int orc_slot_weights(const double* u, double* g) {
  slot_softmax(u, g);
  return 0;
}

/* MLP of one primitive on one encoded input: raw outputs, for tests. */
int orc_mlp(const orc_cfg* cfg, const double* w, const double* enc, double* out) {
  if (!cfg_valid(cfg)) return -1;
  model_t m;
  model_init(&m, cfg);
  double* acts = (double*)malloc(sizeof(double) * (size_t)m.act_size);
  if (!acts) return 1;
  memcpy(acts, enc, sizeof(double) * (size_t)m.nin);
  mlp_forward(&m, w, acts);
  memcpy(out, acts + (m.act_size - m.nout), sizeof(double) * (size_t)m.nout);
  free(acts);
  return 0;
}
