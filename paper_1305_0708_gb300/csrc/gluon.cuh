// All-gluon processes g g > g ... g: colour-ordered sub-currents run by one
// thread block per event, and the colour sum over the (n-1)! orderings.
//
// Tables (generated by the process compiler, gluon_tables<N>.h): every ordered
// tuple S of the non-root legs is a current, built from its consecutive
// splittings with the colour-ordered three- and four-gluon vertices; the
// amplitude of ordering s contracts the root's polarisation with the amputated
// current of the whole tuple.  The exact colour matrix over the traces
// Tr(t^0 t^s1 ...) comes with a common denominator.
//
// Per event, one block: (1) momenta and 1/P^2 of every current (helicity
// independent); (2) for each helicity of the non-root legs: external
// polarisation vectors, the currents phase by phase (tuple length 2, 3, ...;
// thread i computes current i of the phase), the amplitudes for both root
// helicities, and the colour quadratic form; (3) block sum over helicities.
#pragma once
#include <cstdint>

#include "heget.cuh"

#ifdef __CUDA_ARCH__
#define ME_GT(name) name
#else
#define ME_GT(name) name##_h
#endif

namespace me {
namespace gluon {

// X^mu of the colour-ordered three-gluon vertex, legs (1, 2, X) in cyclic order, outgoing momenta
template <class R>
__host__ __device__ __forceinline__ W4<R> v3(const W4<R>& J1, P4<R> k1, const W4<R>& J2, P4<R> k2) {
  const P4<R> kx = {-(k1.e + k2.e), -(k1.x + k2.x), -(k1.y + k2.y), -(k1.z + k2.z)};
  const P4<R> d12 = {k1.e - k2.e, k1.x - k2.x, k1.y - k2.y, k1.z - k2.z};
  const P4<R> d2x = {k2.e - kx.e, k2.x - kx.x, k2.y - kx.y, k2.z - kx.z};
  const P4<R> dx1 = {kx.e - k1.e, kx.x - k1.x, kx.y - k1.y, kx.z - k1.z};
  const cx<R> j12 = mdot(J1, J2), a = mdot(d2x, J1), b = mdot(dx1, J2);
  W4<R> o;
  o.c[0] = d12.e * j12 + J2.c[0] * a + J1.c[0] * b;
  o.c[1] = d12.x * j12 + J2.c[1] * a + J1.c[1] * b;
  o.c[2] = d12.y * j12 + J2.c[2] * a + J1.c[2] * b;
  o.c[3] = d12.z * j12 + J2.c[3] * a + J1.c[3] * b;
  return o;
}

// colour-ordered four-gluon contraction, legs (1, 2, 3, X): 2 (J1.J3) J2 - (J1.J2) J3 - (J2.J3) J1
template <class R>
__host__ __device__ __forceinline__ W4<R> v4(const W4<R>& J1, const W4<R>& J2, const W4<R>& J3) {
  const cx<R> a = mdot(J1, J3), b = mdot(J1, J2), c = mdot(J2, J3);
  const cx<R> a2 = a + a;
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = a2 * J2.c[k] - b * J3.c[k] - c * J1.c[k];
  return o;
}

template <class R>
__host__ __device__ __forceinline__ void acc(W4<R>& s, const W4<R>& t, R f) {
#pragma unroll
  for (int k = 0; k < 4; ++k) s.c[k] = s.c[k] + f * t.c[k];
}

// Sum of the vertex terms of one table entry (amputated, without 1/P^2).
template <class R>
__host__ __device__ __forceinline__ W4<R> entry_sum(const int32_t* meta, const int16_t* terms, const W4<R>* J,
                                                    const P4<R>* K, R g, R g2) {
  const int nv3 = meta[1], nv4 = meta[2], off = meta[3];
  W4<R> s;
#pragma unroll
  for (int k = 0; k < 4; ++k) s.c[k] = mk(R(0), R(0));
  int t = off;
  for (int i = 0; i < nv3; ++i, t += 2) {
    const int a = terms[t], b = terms[t + 1];
    acc(s, v3(J[a], K[a], J[b], K[b]), g);
  }
  for (int i = 0; i < nv4; ++i, t += 3) {
    acc(s, v4(J[terms[t]], J[terms[t + 1]], J[terms[t + 2]]), g2);
  }
  return s;
}

}  // namespace gluon
}  // namespace me
