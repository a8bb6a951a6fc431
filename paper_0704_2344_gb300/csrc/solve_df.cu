// Instantiates the persistent solve kernels (single system and jobs) for
// FP32-pair products; one translation unit per product arithmetic.
#include "solve_kernels.cuh"

namespace fe {
template fe_status dispatch<DFloat>(fe_ctx*, int, SolveParams&);
template fe_status launch_jobs_w<DFloat>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);
}  // namespace fe
