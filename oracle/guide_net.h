// Internal interface of the FP64 guide network (guide_oracle.cpp) for the
// oracle's guided path tracer (oracle.cpp).  TEST INFRASTRUCTURE ONLY: part of
// the CPU oracle, shared by its two files and by nothing else.
#ifndef ORACLE_GUIDE_NET_H
#define ORACLE_GUIDE_NET_H

#include <cstdint>

namespace oguide {

constexpr int kLobes = 8;

// Network parameters and encoding of one scene (a copy of the caller's data).
struct Net;

// grid [8][2^log2_T][4] and W (W1 | W2 | W3 | W4, row-major [in][out]) as
// floats; bf16_act: layer inputs rounded to BF16 (the BF16 network).
Net* net_create(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max, const float* grid,
                const float* W, int bf16_act);
void net_destroy(Net* net);

// The 48 head outputs Y at position p, normal n, band group g.
void net_outputs(const Net* net, const double p[3], const double n[3], uint32_t group, double Y[48]);

// The von Mises-Fisher mixture of head outputs Y: lobe weights (softmax),
// unit mean directions and concentrations kappa = 0.5 + softplus.
struct Mixture {
  double pi[kLobes];
  double mu[kLobes][3];
  double kappa[kLobes];
};
void mixture_of(const double Y[48], Mixture* m);
// Mixture density q(w) at the unit direction w (per steradian).
double mixture_density(const Mixture& m, const double w[3]);

}  // namespace oguide

#endif
