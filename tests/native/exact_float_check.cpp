// Reads hex doubles, prints mg_to_float of each as the FP32 bit pattern, and
// for pairs "F emax x" the round trip mg_unfix(mg_fix(x, emax)).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_1901_11370_gb300/csrc/mg_exact.h"

int main() {
    char tag[8], buf[64];
    while (std::scanf("%7s", tag) == 1) {
        if (tag[0] == 'W') {  // FP32 bit pattern in hex -> FP64 hex float
            unsigned u;
            if (std::scanf("%x", &u) != 1) return 1;
            float f;
            std::memcpy(&f, &u, 4);
            std::printf("%a\n", mg::mg_from_float(f));
        } else if (tag[0] == 'C') {
            if (std::scanf("%63s", buf) != 1) return 1;
            float f = mg::mg_to_float(std::strtod(buf, nullptr));
            unsigned u;
            std::memcpy(&u, &f, 4);
            std::printf("%08x\n", u);
        } else {
            int em;
            if (std::scanf("%d %63s", &em, buf) != 2) return 1;
            double out = 0;
            bool ok = mg::mg_unfix(mg::mg_fix(std::strtod(buf, nullptr), em), em, out);
            if (ok) std::printf("%a\n", out);
            else std::printf("fallback\n");
        }
    }
    return 0;
}
