// serve.cpp -- placeholder until the serving loop lands.
#include "ctx_internal.h"

namespace rxgs {
struct ServeState {};
void destroy_serve(ServeState* s) { delete s; }
}  // namespace rxgs
