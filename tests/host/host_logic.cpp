// Host-side inline logic of the crowd library, compiled without a GPU by
// tests/test_host_logic.py: prints choose_tile and episode_restart results
// for the cases the test names on its command line.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "crowd_internal.h"

int main(int argc, char** argv) {
    for (int k = 1; k + 1 < argc; k += 2) {
        if (!std::strcmp(argv[k], "tile")) {
            int n, W, H;
            if (std::sscanf(argv[k + 1], "%d,%d,%d", &n, &W, &H) != 3) return 2;
            int tx = 0, ty = 0;
            crowd::choose_tile(n, W, H, tx, ty);
            std::printf("tile %d %d\n", tx, ty);
        } else if (!std::strcmp(argv[k], "restart")) {
            int L;
            long long step, origin;
            if (std::sscanf(argv[k + 1], "%d,%lld,%lld", &L, &step, &origin) != 3) return 2;
            std::printf("restart %d\n", crowd::episode_restart(L, step, origin) ? 1 : 0);
        } else {
            return 2;
        }
    }
    return 0;
}
