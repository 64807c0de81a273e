// step1d_inst.cu -- explicit instances of the fused 1D step kernel
// (step1d_kernel.cuh).  The build compiles this unit once per variant with
// SHE_V_REAL (float|double), SHE_V_DIR, SHE_V_SP, SHE_V_PC and SHE_V_VAR
// (0|1) defined, so that the variants compile in parallel; compiled without
// them it instantiates every variant.  The material table (VAR) is for heat
// rods only.  With SHE_V_IMP = 1 the unit holds the implicit-scheme kernel of
// (SHE_V_REAL, SHE_V_DIR, SHE_V_SP) instead.
#include "step1d_kernel.cuh"

namespace she {

#if defined(SHE_V_REAL) && defined(SHE_V_IMP) && SHE_V_IMP
template cudaError_t launch_step1d_theta<SHE_V_REAL, (bool)SHE_V_DIR, (bool)SHE_V_SP>(const Step1DArgs<SHE_V_REAL>&,
                                                                                   int, cudaStream_t);
#elif defined(SHE_V_REAL)
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
#define SHE_STEP1D_THETA(R, D, S) \
    template cudaError_t launch_step1d_theta<R, D, S>(const Step1DArgs<R>&, int, cudaStream_t);
SHE_STEP1D_THETA(float, false, false)
SHE_STEP1D_THETA(float, false, true)
SHE_STEP1D_THETA(float, true, false)
SHE_STEP1D_THETA(float, true, true)
SHE_STEP1D_THETA(double, false, false)
SHE_STEP1D_THETA(double, false, true)
SHE_STEP1D_THETA(double, true, false)
SHE_STEP1D_THETA(double, true, true)
#undef SHE_STEP1D_THETA
#undef SHE_STEP1D_INST_DSP
#undef SHE_STEP1D_INST
#endif

}  // namespace she
