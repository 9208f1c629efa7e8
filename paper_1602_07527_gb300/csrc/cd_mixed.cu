// Mixed-precision engine (split-BF16 operands on tcgen05 tensor cores).
#include "cd_internal.h"
#include "cd_mixed.h"

namespace cd {
int mixed_init() { return CD_OK; }
bool mixed_available() { return false; }
size_t mixed_workspace_bytes(int, int, int) { return 0; }
}  // namespace cd
