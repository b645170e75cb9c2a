// Gauss-Newton refinement and adjoint gradient (placeholder translation unit).
#include "cdc_host.h"
