// Host-side test of the work-buffer arena of the CUDA library (no GPU needed): carves are 256-byte
// aligned and stay inside the buffer; a carve past the end, a missing buffer or a size that would
// wrap returns NULL and sets the overflow flag for good, and Arena::check then reports
// DBI_ERR_WORKSPACE with a message naming the caller.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_2402_02116_gb300/csrc/common.cuh"

static int fails = 0;
#define EXPECT(c)                                                   \
  do {                                                              \
    if (!(c)) {                                                     \
      std::fprintf(stderr, "line %d: expected %s\n", __LINE__, #c); \
      ++fails;                                                      \
    }                                                               \
  } while (0)

int main() {
  using dbi::Arena;
  std::vector<unsigned char> buf(4096 + 256);
  char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(buf.data()) + 255) & ~uintptr_t(255));
  {
    Arena ar(base, 4096);
    char *a = static_cast<char *>(ar.take(1));
    char *b = static_cast<char *>(ar.take(300));
    char *c = static_cast<char *>(ar.take(256));
    EXPECT(a == base && b == base + 256 && c == base + 768);
    EXPECT(!ar.overflow && ar.check("fits") == DBI_OK);
    char *d = static_cast<char *>(ar.take(4096 - 1024));  // exactly to the end
    EXPECT(d == base + 1024 && !ar.overflow && ar.used == 4096);
    EXPECT(ar.take(1) == nullptr && ar.overflow);
    EXPECT(ar.take(0) == nullptr);  // nothing is handed out after an overflow
    EXPECT(ar.check("carve_test") == DBI_ERR_WORKSPACE);
    EXPECT(std::strstr(dbi_last_error(), "carve_test") != nullptr);
  }
  {
    Arena ar(base, 4096);
    EXPECT(ar.take(5000) == nullptr && ar.overflow);
    EXPECT(ar.take(16) == nullptr);
  }
  {
    Arena ar(nullptr, 1 << 20);
    EXPECT(ar.take(16) == nullptr && ar.overflow && ar.check("null") == DBI_ERR_WORKSPACE);
  }
  {
    Arena ar(base, 4096);
    EXPECT(ar.take(256) == base);
    EXPECT(ar.take(SIZE_MAX - 10) == nullptr && ar.overflow);  // the aligned size would wrap
    EXPECT(ar.take(SIZE_MAX / 2) == nullptr);
  }
  if (fails) return 1;
  std::puts("arena ok");
  return 0;
}
