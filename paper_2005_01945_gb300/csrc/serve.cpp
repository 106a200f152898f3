// serve.cpp -- placeholder until the serving loop lands.
#include "runtime.h"
namespace tgb {
void release_serving(tfhe_ctx *) {}
}  // namespace tgb
