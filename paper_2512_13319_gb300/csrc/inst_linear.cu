// One explicit instance of the linear-model solver; the build compiles this
// file once per (INST_N, INST_M, INST_S) so the instances build in parallel.
#include "solve_impl.cuh"
namespace mapk {
template const Ops* linear_ops<INST_N, INST_M, INST_S>();
}  // namespace mapk
