// lmfmm_mixed.cu -- mixed-precision apply path (filled in below).
#include "internal.h"
