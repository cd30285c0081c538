"""FP64 CPU oracle of the electron-swarm step loop (test infrastructure only)."""
