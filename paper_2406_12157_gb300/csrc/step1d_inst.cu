// step1d_inst.cu -- explicit instances of the fused 1D step kernel
// (step1d_kernel.cuh).  The build compiles this unit once per variant with
// SHE_V_REAL (float|double), SHE_V_DIR, SHE_V_SP, SHE_V_PC and SHE_V_VAR
// (0|1) defined, so that the variants compile in parallel; compiled without
// them it instantiates every variant.  The material table (VAR) is for heat
// rods only.
#include "step1d_kernel.cuh"

namespace she {

#if defined(SHE_V_REAL)
template cudaError_t launch_step1d_variant<SHE_V_REAL, (bool)SHE_V_DIR, (bool)SHE_V_SP, (bool)SHE_V_PC,
                                           (bool)SHE_V_VAR>(const Step1DArgs<SHE_V_REAL>&, int, cudaStream_t);
#else
#define SHE_STEP1D_INST(R, D, S, P, V) \
    template cudaError_t launch_step1d_variant<R, D, S, P, V>(const Step1DArgs<R>&, int, cudaStream_t);
#define SHE_STEP1D_INST_DSP(R, P)                \
    SHE_STEP1D_INST(R, false, false, P, false)   \
    SHE_STEP1D_INST(R, false, true, P, false)    \
    SHE_STEP1D_INST(R, true, false, P, false)    \
    SHE_STEP1D_INST(R, true, true, P, false)     \
    SHE_STEP1D_INST(R, false, false, P, true)    \
    SHE_STEP1D_INST(R, true, false, P, true)
SHE_STEP1D_INST_DSP(float, false)
SHE_STEP1D_INST_DSP(float, true)
SHE_STEP1D_INST_DSP(double, false)
SHE_STEP1D_INST_DSP(double, true)
#undef SHE_STEP1D_INST_DSP
#undef SHE_STEP1D_INST
#endif

}  // namespace she
