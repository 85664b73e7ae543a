// Mixed-precision correction solve (filled in by the FP32 operator work).
#include "mk_device.cuh"

namespace mk {

int solve_mixed(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, double sigma, const double* rhs,
                const double*, const double*, double* x, int ld, int N, const mk_solve_opts& o, mk_solve_report* rep,
                cudaStream_t s) {
  (void)ctx; (void)m; (void)mol; (void)sigma; (void)rhs; (void)x; (void)ld; (void)N; (void)o; (void)rep; (void)s;
  return fail(MK_ERR_UNSUPPORTED, "mixed precision not built yet");
}

}  // namespace mk
