// Error reporting and version of the C ABI.
#include <cstring>

#include "common.h"

namespace mrf {
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
}  // namespace mrf

extern "C" const char* mrf_last_error(void) { return mrf::g_err; }
extern "C" int mrf_abi_version(void) { return 1; }
