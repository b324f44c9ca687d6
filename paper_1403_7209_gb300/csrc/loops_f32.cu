// FP32-arithmetic edge loops of the mixed path: Green-Gauss (FP32 sums),
// first- and second-order flux (each edge's FP32 flux is converted to FP64
// before it is added into the FP64 residual).
#include "gg_gather.cuh"
#include "launch.cuh"

namespace op2b {

int launch_f32(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  Gas<float> g{(float)L.gamma, (float)(L.gamma - 1.0), (float)L.eps, (float)(2.0 * L.eps)};
  switch (L.loop) {
    case OP2B_LOOP_GREEN_GAUSS: {
      if (s.strategy == OP2B_STRAT_GATHER) return launch_gg_gather<float, 2>(c, L, s.block);
      BodyGG<float> b{(const float*)L.q, L.ldq, (const float*)L.n, L.ldn};
      Targets<float, 18> tg{(float*)L.t0, L.ldt0, (float*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX1: {
      BodyFlux1<float> b{(const float*)L.q, L.ldq, (const float*)L.n, L.ldn, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    case OP2B_LOOP_FLUX2: {
      BodyFlux2<float> b{(const float*)L.q, L.ldq, (const float*)L.G, L.ldG,
                         (const float*)L.n, L.ldn, (const float*)L.dx, L.lddx, g};
      Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
      return run_body(c, b, L, s, tg);
    }
    default:
      return c->fail(OP2B_EINVAL, "launch_f32: loop has no FP32 variant");
  }
}

}  // namespace op2b
