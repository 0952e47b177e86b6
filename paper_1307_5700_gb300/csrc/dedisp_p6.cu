// Dedispersion kernel instantiations (A5, Sec. 2.2.2): the shapes whose
// index is 6 modulo kDedispParts.
#define TP_DEDISP_PART 6
#include "dedisp_kernel.cuh"

TP_DEFINE_DEDISP_PART(6)
