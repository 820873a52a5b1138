// CPU FP64 oracle of the learned path guide (test infrastructure only).
//
// The guide proposes directions at Lambertian vertices, mixed with cosine
// sampling by one-sample MIS (it replaces nothing in the estimator of
// section 4, Eq. 2; it only changes the sampling density).  Its definition,
// written here plainly in double precision, is:
//
//   input (64):  multiresolution hash-grid encoding of the position (8
//                levels x 4 features, trilinear; after Mueller et al. 2022,
//                spatial hash with primes 1, 2654435761, 805459861), real
//                spherical harmonics of the normal up to degree 3 (16), a
//                one-hot band group (9), zeros (7);
//   MLP:         64 -> 64 -> 64 -> 64 -> 48, ReLU on the hidden layers, no
//                biases;
//   head:        8 von Mises-Fisher lobes from outputs 5j..5j+4: softmax
//                weight, mean direction m / |m|, kappa = 0.5 + softplus;
//   density:     q(w) = sum_j pi_j kappa_j / (2 pi (1 - e^{-2 kappa_j}))
//                       exp(kappa_j (mu_j . w - 1));
//   loss:        L = -(1/N) sum_r (w_r / mean(w)) log q_r(omega_r),
//                w_r = incident radiance x cosine / sampling pdf of record r;
//   gradients:   by the chain rule through head, MLP and the trilinear
//                interpolation of the grid.
//
// The network runs in BF16 with FP32 accumulation: with bf16_act the oracle
// rounds every layer input (X, H1, H2, H3) to BF16 as that definition says and
// accumulates in FP64; without it the activations are exact (the form the
// finite-difference pins check).  Weights arrive as floats (BF16-rounded by
// the caller when comparing with the GPU).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "guide_net.h"

namespace {

constexpr int kLevels = 8, kFeat = 4, kIn = 64, kHid = 64, kOut = 48, kLobes = 8, kGroups = 9;

struct GCfg {
  uint32_t log2_T;
  double lo[3], hi[3];
  std::vector<uint32_t> res;  // per level
};

// real spherical harmonics, degree <= 3, of a unit vector
void sh16(double x, double y, double z, double* o) {
  const double pi = M_PI;
  const double c0 = 0.5 / std::sqrt(pi);
  const double c1 = std::sqrt(3.0) / (2.0 * std::sqrt(pi));
  const double c2 = std::sqrt(15.0) / (2.0 * std::sqrt(pi));
  const double c3 = std::sqrt(5.0) / (4.0 * std::sqrt(pi));
  const double c4 = std::sqrt(15.0) / (4.0 * std::sqrt(pi));
  const double c5 = std::sqrt(35.0 / (2.0 * pi)) / 4.0;
  const double c6 = std::sqrt(105.0) / (2.0 * std::sqrt(pi));
  const double c7 = std::sqrt(21.0 / (2.0 * pi)) / 4.0;
  const double c8 = std::sqrt(7.0) / (4.0 * std::sqrt(pi));
  const double c9 = std::sqrt(105.0) / (4.0 * std::sqrt(pi));
  o[0] = c0;
  o[1] = -c1 * y;
  o[2] = c1 * z;
  o[3] = -c1 * x;
  o[4] = c2 * x * y;
  o[5] = -c2 * y * z;
  o[6] = c3 * (3.0 * z * z - 1.0);
  o[7] = -c2 * x * z;
  o[8] = c4 * (x * x - y * y);
  o[9] = -c5 * y * (3.0 * x * x - y * y);
  o[10] = c6 * x * y * z;
  o[11] = -c7 * y * (5.0 * z * z - 1.0);
  o[12] = c8 * z * (5.0 * z * z - 3.0);
  o[13] = -c7 * x * (5.0 * z * z - 1.0);
  o[14] = c9 * z * (x * x - y * y);
  o[15] = -c5 * x * (x * x - 3.0 * y * y);
}

// grid vertex index of level l (dense when the level fits the table)
uint32_t grid_index(const GCfg& g, int l, uint32_t cx, uint32_t cy, uint32_t cz) {
  const uint32_t T = 1u << g.log2_T;
  const uint64_t r1 = (uint64_t)g.res[l] + 1;
  if (r1 * r1 * r1 <= T) return (uint32_t)(cx + cy * r1 + cz * r1 * r1);
  return (cx * 1u ^ cy * 2654435761u ^ cz * 805459861u) & (T - 1u);
}

// One record's corners and weights per level.
struct Enc {
  uint32_t idx[kLevels][8];
  double w[kLevels][8];
};

void encode(const GCfg& g, const float* grid, const double p[3], const double n[3], uint32_t group, double* X,
            Enc* e) {
  double u[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = (p[a] - g.lo[a]) / (g.hi[a] - g.lo[a]);
    u[a] = u[a] < 0.0 ? 0.0 : (u[a] > 1.0 ? 1.0 : u[a]);
  }
  const uint32_t T = 1u << g.log2_T;
  for (int l = 0; l < kLevels; ++l) {
    uint32_t c[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      const double s = u[a] * g.res[l];
      double fl = std::floor(s);
      if (fl > g.res[l] - 1) fl = g.res[l] - 1;
      c[a] = (uint32_t)fl;
      f[a] = s - fl;
    }
    double acc[kFeat] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < 8; ++k) {
      const uint32_t dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
      const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
      const uint32_t id = grid_index(g, l, c[0] + dx, c[1] + dy, c[2] + dz);
      e->idx[l][k] = id;
      e->w[l][k] = w;
      for (int q = 0; q < kFeat; ++q) acc[q] += w * (double)grid[((size_t)l * T + id) * kFeat + q];
    }
    for (int q = 0; q < kFeat; ++q) X[kFeat * l + q] = acc[q];
  }
  sh16(n[0], n[1], n[2], X + 32);
  for (int i = 48; i < kIn; ++i) X[i] = 0.0;
  X[48 + group] = 1.0;
}

void matvec(const double* x, const float* W, int in, int out, double* y) {
  for (int o = 0; o < out; ++o) y[o] = 0.0;
  for (int i = 0; i < in; ++i)
    for (int o = 0; o < out; ++o) y[o] += x[i] * (double)W[(size_t)i * out + o];
}

double softplus(double x) { return x > 30.0 ? x : std::log1p(std::exp(x)); }

// BF16 network: with bf16_act the inputs of every layer (X, H1, H2, H3) are
// rounded to BF16 (round to nearest even of the float value) before the
// product; gradients pass through the rounding unchanged.
double round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

void maybe_round(double* v, int n, int on) {
  if (on)
    for (int i = 0; i < n; ++i) v[i] = round_bf16(v[i]);
}
double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }

struct Head {
  double pi[kLobes], mu[kLobes][3], kappa[kLobes], mnorm[kLobes];
};

void head(const double* Y, Head* h) {
  double mx = -INFINITY;
  for (int j = 0; j < kLobes; ++j) mx = std::fmax(mx, Y[5 * j]);
  double s = 0.0;
  for (int j = 0; j < kLobes; ++j) {
    h->pi[j] = std::exp(Y[5 * j] - mx);
    s += h->pi[j];
  }
  for (int j = 0; j < kLobes; ++j) {
    h->pi[j] /= s;
    const double m0 = Y[5 * j + 1], m1 = Y[5 * j + 2], m2 = Y[5 * j + 3];
    double nm = std::sqrt(m0 * m0 + m1 * m1 + m2 * m2);
    if (nm < 1e-6) nm = 1e-6;
    h->mnorm[j] = nm;
    h->mu[j][0] = m0 / nm;
    h->mu[j][1] = m1 / nm;
    h->mu[j][2] = m2 / nm;
    h->kappa[j] = 0.5 + softplus(Y[5 * j + 4]);
  }
}

double vmf(double kappa, const double mu[3], const double w[3]) {
  const double c = mu[0] * w[0] + mu[1] * w[1] + mu[2] * w[2];
  return kappa / (2.0 * M_PI * (-std::expm1(-2.0 * kappa))) * std::exp(kappa * (c - 1.0));
}

GCfg make_cfg(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max) {
  GCfg g;
  g.log2_T = log2_T;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = lo[a];
    g.hi[a] = hi[a];
  }
  const double b = std::exp((std::log((double)n_max) - std::log((double)n_min)) / (kLevels - 1));
  g.res.resize(kLevels);
  // n_min b^l rounded down; the relative 1e-12 keeps a product that is an
  // integer in exact arithmetic (16 x 2^7 = 2048) from landing just below it
  for (int l = 0; l < kLevels; ++l) g.res[l] = (uint32_t)std::floor((double)n_min * std::pow(b, l) * (1.0 + 1e-12));
  return g;
}

}  // namespace

extern "C" {

// Per-level grid resolutions used by the encoding.
void or_guide_resolutions(float n_min, float n_max, uint32_t* res) {
  const float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  GCfg g = make_cfg(19, lo, hi, n_min, n_max);
  for (int l = 0; l < kLevels; ++l) res[l] = g.res[l];
}

// Forward pass for n records: X [n][64], Y [n][48], q(omega) [n].
// W = W1 [64][64] | W2 [64][64] | W3 [64][64] | W4 [64][48], row-major [in][out].
void or_guide_forward(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max, const float* grid,
                      const float* W, uint64_t n, const float* pos, const float* nrm, const uint32_t* group,
                      const float* omega, int bf16_act, double* X_out, double* Y_out, double* q_out) {
  const GCfg g = make_cfg(log2_T, lo, hi, n_min, n_max);
  const float* W1 = W;
  const float* W2 = W1 + kIn * kHid;
  const float* W3 = W2 + kHid * kHid;
  const float* W4 = W3 + kHid * kHid;
  std::vector<Enc> enc(1);
  for (uint64_t r = 0; r < n; ++r) {
    double p[3] = {pos[3 * r], pos[3 * r + 1], pos[3 * r + 2]};
    double nn[3] = {nrm[3 * r], nrm[3 * r + 1], nrm[3 * r + 2]};
    double X[kIn], H1[kHid], H2[kHid], H3[kHid], Y[kOut];
    encode(g, grid, p, nn, group[r], X, &enc[0]);
    maybe_round(X, kIn, bf16_act);
    matvec(X, W1, kIn, kHid, H1);
    for (double& v : H1) v = v > 0.0 ? v : 0.0;
    maybe_round(H1, kHid, bf16_act);
    matvec(H1, W2, kHid, kHid, H2);
    for (double& v : H2) v = v > 0.0 ? v : 0.0;
    maybe_round(H2, kHid, bf16_act);
    matvec(H2, W3, kHid, kHid, H3);
    for (double& v : H3) v = v > 0.0 ? v : 0.0;
    maybe_round(H3, kHid, bf16_act);
    matvec(H3, W4, kHid, kOut, Y);
    if (X_out) std::memcpy(X_out + r * kIn, X, sizeof(X));
    if (Y_out) std::memcpy(Y_out + r * kOut, Y, sizeof(Y));
    if (q_out) {
      Head h;
      head(Y, &h);
      double w[3] = {omega[3 * r], omega[3 * r + 1], omega[3 * r + 2]};
      double q = 0.0;
      for (int j = 0; j < kLobes; ++j) q += h.pi[j] * vmf(h.kappa[j], h.mu[j], w);
      q_out[r] = q;
    }
  }
}

// Loss and gradients for n records with weights wt (>= 0).
// dW (same layout as W) and dgrid ([8 * T * 4]) are overwritten.
double or_guide_loss_grad(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max,
                          const float* grid, const float* W, uint64_t n, const float* pos, const float* nrm,
                          const uint32_t* group, const float* omega, const float* wt, int bf16_act, double* dW,
                          double* dgrid) {
  const GCfg g = make_cfg(log2_T, lo, hi, n_min, n_max);
  const uint32_t T = 1u << log2_T;
  const float* W1 = W;
  const float* W2 = W1 + kIn * kHid;
  const float* W3 = W2 + kHid * kHid;
  const float* W4 = W3 + kHid * kHid;
  double* dW1 = dW;
  double* dW2 = dW1 + kIn * kHid;
  double* dW3 = dW2 + kHid * kHid;
  double* dW4 = dW3 + kHid * kHid;
  std::memset(dW, 0, sizeof(double) * (kIn * kHid + 2 * kHid * kHid + kHid * kOut));
  std::memset(dgrid, 0, sizeof(double) * (size_t)kLevels * T * kFeat);
  double wsum = 0.0;
  for (uint64_t r = 0; r < n; ++r) wsum += wt[r];
  if (!(wsum > 0.0) || n == 0) return 0.0;
  const double wbar = wsum / (double)n;
  double loss = 0.0;
  Enc e;
  for (uint64_t r = 0; r < n; ++r) {
    double p[3] = {pos[3 * r], pos[3 * r + 1], pos[3 * r + 2]};
    double nn[3] = {nrm[3 * r], nrm[3 * r + 1], nrm[3 * r + 2]};
    double w[3] = {omega[3 * r], omega[3 * r + 1], omega[3 * r + 2]};
    double X[kIn], Z1[kHid], H1[kHid], Z2[kHid], H2[kHid], Z3[kHid], H3[kHid], Y[kOut];
    encode(g, grid, p, nn, group[r], X, &e);
    maybe_round(X, kIn, bf16_act);
    matvec(X, W1, kIn, kHid, Z1);
    for (int i = 0; i < kHid; ++i) H1[i] = Z1[i] > 0.0 ? Z1[i] : 0.0;
    maybe_round(H1, kHid, bf16_act);
    matvec(H1, W2, kHid, kHid, Z2);
    for (int i = 0; i < kHid; ++i) H2[i] = Z2[i] > 0.0 ? Z2[i] : 0.0;
    maybe_round(H2, kHid, bf16_act);
    matvec(H2, W3, kHid, kHid, Z3);
    for (int i = 0; i < kHid; ++i) H3[i] = Z3[i] > 0.0 ? Z3[i] : 0.0;
    maybe_round(H3, kHid, bf16_act);
    matvec(H3, W4, kHid, kOut, Y);
    Head h;
    head(Y, &h);
    double pj[kLobes], q = 0.0;
    for (int j = 0; j < kLobes; ++j) {
      pj[j] = vmf(h.kappa[j], h.mu[j], w);
      q += h.pi[j] * pj[j];
    }
    const double a = wt[r] / (wbar * (double)n);  // this record's factor in L
    loss -= a * std::log(q);
    // dL/dY = -a * d log q / dY
    double dY[kOut] = {0};
    for (int j = 0; j < kLobes; ++j) {
      const double rj = h.pi[j] * pj[j] / q;
      const double c = h.mu[j][0] * w[0] + h.mu[j][1] * w[1] + h.mu[j][2] * w[2];
      dY[5 * j] = -a * (rj - h.pi[j]);
      for (int d = 0; d < 3; ++d)
        dY[5 * j + 1 + d] = -a * rj * h.kappa[j] * (w[d] - c * h.mu[j][d]) / h.mnorm[j];
      const double k = h.kappa[j];
      const double dlogp = 1.0 / k - 2.0 / std::expm1(2.0 * k) + (c - 1.0);
      dY[5 * j + 4] = -a * rj * dlogp * sigmoid(Y[5 * j + 4]);
    }
    // backward through the MLP
    double dH3[kHid], dZ3[kHid], dH2[kHid], dZ2[kHid], dH1[kHid], dZ1[kHid], dX[kIn];
    for (int i = 0; i < kHid; ++i) {
      double s = 0.0;
      for (int o = 0; o < kOut; ++o) s += dY[o] * (double)W4[i * kOut + o];
      dH3[i] = s;
      for (int o = 0; o < kOut; ++o) dW4[i * kOut + o] += H3[i] * dY[o];
    }
    for (int i = 0; i < kHid; ++i) dZ3[i] = Z3[i] > 0.0 ? dH3[i] : 0.0;
    for (int i = 0; i < kHid; ++i) {
      double s = 0.0;
      for (int o = 0; o < kHid; ++o) s += dZ3[o] * (double)W3[i * kHid + o];
      dH2[i] = s;
      for (int o = 0; o < kHid; ++o) dW3[i * kHid + o] += H2[i] * dZ3[o];
    }
    for (int i = 0; i < kHid; ++i) dZ2[i] = Z2[i] > 0.0 ? dH2[i] : 0.0;
    for (int i = 0; i < kHid; ++i) {
      double s = 0.0;
      for (int o = 0; o < kHid; ++o) s += dZ2[o] * (double)W2[i * kHid + o];
      dH1[i] = s;
      for (int o = 0; o < kHid; ++o) dW2[i * kHid + o] += H1[i] * dZ2[o];
    }
    for (int i = 0; i < kHid; ++i) dZ1[i] = Z1[i] > 0.0 ? dH1[i] : 0.0;
    for (int i = 0; i < kIn; ++i) {
      double s = 0.0;
      for (int o = 0; o < kHid; ++o) s += dZ1[o] * (double)W1[i * kHid + o];
      dX[i] = s;
      for (int o = 0; o < kHid; ++o) dW1[i * kHid + o] += X[i] * dZ1[o];
    }
    for (int l = 0; l < kLevels; ++l)
      for (int k = 0; k < 8; ++k)
        for (int f = 0; f < kFeat; ++f) dgrid[((size_t)l * T + e.idx[l][k]) * kFeat + f] += e.w[l][k] * dX[kFeat * l + f];
  }
  return loss;
}

// One Adam step (Kingma and Ba, 2015) on n parameters in place: first and
// second moment estimates m, v with decay rates b1, b2, bias-corrected by
// 1 - b^t for step t >= 1, then p -= lr m_hat / (sqrt(v_hat) + eps).
void or_adam_step(uint64_t n, double* p, const double* g, double* m, double* v, double lr, double b1, double b2,
                  double eps, uint32_t t) {
  const double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
  for (uint64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

// Mixture density of given head outputs Y [48] at n directions (for
// quadrature checks of the normalisation).
void or_guide_density(const double* Y, uint64_t n, const double* omega, double* q) {
  Head h;
  head(Y, &h);
  for (uint64_t r = 0; r < n; ++r) {
    double w[3] = {omega[3 * r], omega[3 * r + 1], omega[3 * r + 2]};
    double s = 0.0;
    for (int j = 0; j < kLobes; ++j) s += h.pi[j] * vmf(h.kappa[j], h.mu[j], w);
    q[r] = s;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// the network as an object, for the guided path tracer of oracle.cpp
// ---------------------------------------------------------------------------
namespace oguide {

struct Net {
  GCfg g;
  std::vector<float> grid, W;
  int bf16_act;
};

Net* net_create(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max, const float* grid,
                const float* W, int bf16_act) {
  Net* net = new Net();
  net->g = make_cfg(log2_T, lo, hi, n_min, n_max);
  net->grid.assign(grid, grid + (size_t)kLevels * (1u << log2_T) * kFeat);
  net->W.assign(W, W + (kIn * kHid + 2 * kHid * kHid + kHid * kOut));
  net->bf16_act = bf16_act;
  return net;
}

void net_destroy(Net* net) { delete net; }

void net_outputs(const Net* net, const double p[3], const double n[3], uint32_t group, double Y[48]) {
  const float* W1 = net->W.data();
  const float* W2 = W1 + kIn * kHid;
  const float* W3 = W2 + kHid * kHid;
  const float* W4 = W3 + kHid * kHid;
  double X[kIn], H1[kHid], H2[kHid], H3[kHid];
  Enc e;
  encode(net->g, net->grid.data(), p, n, group, X, &e);
  maybe_round(X, kIn, net->bf16_act);
  matvec(X, W1, kIn, kHid, H1);
  for (double& v : H1) v = v > 0.0 ? v : 0.0;
  maybe_round(H1, kHid, net->bf16_act);
  matvec(H1, W2, kHid, kHid, H2);
  for (double& v : H2) v = v > 0.0 ? v : 0.0;
  maybe_round(H2, kHid, net->bf16_act);
  matvec(H2, W3, kHid, kHid, H3);
  for (double& v : H3) v = v > 0.0 ? v : 0.0;
  maybe_round(H3, kHid, net->bf16_act);
  matvec(H3, W4, kHid, kOut, Y);
}

void mixture_of(const double Y[48], Mixture* m) {
  Head h;
  head(Y, &h);
  for (int j = 0; j < kLobes; ++j) {
    m->pi[j] = h.pi[j];
    m->kappa[j] = h.kappa[j];
    for (int d = 0; d < 3; ++d) m->mu[j][d] = h.mu[j][d];
  }
}

double mixture_density(const Mixture& m, const double w[3]) {
  double s = 0.0;
  for (int j = 0; j < kLobes; ++j) s += m.pi[j] * vmf(m.kappa[j], m.mu[j], w);
  return s;
}

}  // namespace oguide
