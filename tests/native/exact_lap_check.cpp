// Reads lines "M x0 x1 ... xM" (hex floats), prints exact_lap's result as a
// hex float, or "fallback" when it declines.  Built by the CPU test with g++
// against the library's header.
#include <cstdio>
#include <cstdlib>

#include "../../paper_1901_11370_gb300/csrc/mg_exact.h"

int main() {
    int M;
    while (std::scanf("%d", &M) == 1) {
        double v[7];
        for (int j = 0; j <= M; j++) {
            char buf[64];
            if (std::scanf("%63s", buf) != 1) return 1;
            v[j] = std::strtod(buf, nullptr);
        }
        double out = 0;
        bool ok = M == 4 ? mg::exact_lap<4>(v, out) : mg::exact_lap<6>(v, out);
        if (ok) std::printf("%a\n", out);
        else std::printf("fallback\n");
    }
    return 0;
}
