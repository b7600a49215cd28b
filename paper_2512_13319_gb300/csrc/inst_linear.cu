// One explicit instance of the linear-model solver.  The build compiles this
// file twice per (INST_N, INST_M, INST_S), so that the instances build in
// parallel in halves of similar size:
//   INST_PART 0: the operation table, the RTS solve, the chunked batch solve,
//                the cost, the sequential baseline and the occupancy query;
//   INST_PART 1: the two-filter solve, the gradient, the segmented batch solve and
//                the block/exact-element solve with its dense output (state
//                dimensions up to 6), which part 0 declares extern.
#include "solve_impl.cuh"
namespace mapk {
#if INST_PART == 0
#if INST_N <= 6
extern template map_status solve_linear_tf<INST_N, INST_M, INST_S>(map_smoother&, const void*, void*, void*,
                                                                   cudaStream_t, const INST_S*);
extern template map_status grad_linear<INST_N, INST_M, INST_S>(map_smoother&, const void*, const void*,
                                                               const void*, int, double*, cudaStream_t);
extern template map_status solve_linear_seg<INST_N, INST_M, INST_S>(map_smoother&, const void*,
                                                                    const unsigned char*, void*, cudaStream_t);
extern template map_status solve_linear_block<INST_N, INST_M, INST_S>(map_smoother&, const void*, void*, void*,
                                                                      cudaStream_t, bool);
extern template map_status dense_linear<INST_N, INST_M, INST_S>(map_smoother&, const void*, const void*,
                                                                const void*, void*, cudaStream_t);
#endif
template const Ops* linear_ops<INST_N, INST_M, INST_S>();
#else
template map_status solve_linear_tf<INST_N, INST_M, INST_S>(map_smoother&, const void*, void*, void*, cudaStream_t,
                                                            const INST_S*);
template map_status grad_linear<INST_N, INST_M, INST_S>(map_smoother&, const void*, const void*, const void*, int,
                                                        double*, cudaStream_t);
template map_status solve_linear_seg<INST_N, INST_M, INST_S>(map_smoother&, const void*, const unsigned char*,
                                                             void*, cudaStream_t);
template map_status solve_linear_block<INST_N, INST_M, INST_S>(map_smoother&, const void*, void*, void*, cudaStream_t,
                                                               bool);
template map_status dense_linear<INST_N, INST_M, INST_S>(map_smoother&, const void*, const void*, const void*, void*,
                                                         cudaStream_t);
#endif
}  // namespace mapk
