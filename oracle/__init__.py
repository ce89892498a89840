"""CPU FP64 oracle (test infrastructure only; see ddg_oracle's header)."""
