// Serving scheduler of libphasetrack (pt_submit / pt_poll).
#include "pt_internal.h"

extern "C" void pt_serve_shutdown(pt_ctx* c) { (void)c; }
