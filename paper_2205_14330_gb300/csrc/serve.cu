// Serving loop of libpbr (continuous batching of render requests over
// resident scenes).
#include "api_internal.h"

void pbr::serve_shutdown(pbr_ctx *c) { (void)c; }
