// FP64 edge loops: Green-Gauss, first- and second-order flux, spectral radius,
// block-Jacobi blocks.
#include "gg_gather.cuh"
#include "launch.cuh"

namespace op2b {

int launch_f64(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  Gas<double> g{L.gamma, L.gamma - 1.0, L.eps, 2.0 * L.eps};
  switch (L.loop) {
    case OP2B_LOOP_GREEN_GAUSS: {
      if (s.strategy == OP2B_STRAT_GATHER) return launch_gg_gather<double, 2>(c, L, s.block);
      if (s.strategy == OP2B_STRAT_HYBRID) return launch_gg_hybrid(c, L, s.block);
      BodyGG<double> b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn};
      Targets<double, 18> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX1: {
      BodyFlux1<double> b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX2: {
      BodyFlux2<double> b{(const double*)L.q, L.ldq, (const double*)L.G, L.ldG,
                          (const double*)L.n, L.ldn, (const double*)L.dx, L.lddx, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_JACOBI: {
      BodyJacobi b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn, g};
      Targets<double, 36> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_JACOBI_SUMS: {
      BodyJacobiSums b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn, g};
      Targets<double, 4> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_SPECTRAL: {
      BodySpectral b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn, g};
      Targets<double, 1> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    default:
      return c->fail(OP2B_EINVAL, "launch_f64: not an FP64 forward loop");
  }
}

}  // namespace op2b
