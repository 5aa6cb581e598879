// The march instantiations of the denoised chain (gempic_set_denoiser): the same march source
// with its chain hooks compiled in, built as a translation unit of its own so that it compiles
// beside gempic_kernels.cu.  Only the templates and the two entry points below are taken from
// that file here; its other definitions are compiled there.
#define GEMPIC_CHAIN_TU
#include "gempic_kernels.cu"
