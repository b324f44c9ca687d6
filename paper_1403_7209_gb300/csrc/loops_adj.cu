// Derivative edge loops (FP64): adjoint (transposed) and tangent-linear
// flux (first and second order) and Green-Gauss.
#include "launch.cuh"

namespace op2b {

int launch_adj(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  Gas<double> g{L.gamma, L.gamma - 1.0, L.eps, 2.0 * L.eps};
  switch (L.loop) {
    case OP2B_LOOP_FLUX1_ADJ: {
      BodyFluxAdj<1> b{(const double*)L.lam, L.ldl, (const double*)L.q, L.ldq,
                       nullptr, 0, (const double*)L.n, L.ldn, nullptr, 0,
                       (double*)L.direct, L.lddirect, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX2_ADJ: {
      BodyFluxAdj<2> b{(const double*)L.lam, L.ldl, (const double*)L.q, L.ldq,
                       (const double*)L.G, L.ldG, (const double*)L.n, L.ldn,
                       (const double*)L.dx, L.lddx, (double*)L.direct, L.lddirect, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t1, L.ldt1};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_GG_ADJ: {
      BodyGGAdj b{(const double*)L.Gb, L.ldGb, (const double*)L.q, L.ldq,
                  (const double*)L.n, L.ldn, (double*)L.direct, L.lddirect};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_GG_TAN: {
      BodyGGTan b{(const double*)L.q, L.ldq, (const double*)L.qd, L.ldqd,
                  (const double*)L.n, L.ldn, (const double*)L.nd, L.ldnd};
      Targets<double, 18> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX1_TAN: {
      BodyFluxTan<1> b{(const double*)L.q, L.ldq, (const double*)L.qd, L.ldqd, nullptr, 0, nullptr,
                       0, (const double*)L.n, L.ldn, (const double*)L.nd, L.ldnd, nullptr, 0, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX2_TAN: {
      BodyFluxTan<2> b{(const double*)L.q, L.ldq, (const double*)L.qd, L.ldqd,
                       (const double*)L.G, L.ldG, (const double*)L.Gd, L.ldGd,
                       (const double*)L.n, L.ldn, (const double*)L.nd, L.ldnd,
                       (const double*)L.dx, L.lddx, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    default:
      return c->fail(OP2B_EINVAL, "launch_adj: not a derivative loop");
  }
}

}  // namespace op2b
