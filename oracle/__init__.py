"""Independent FP64 oracle of the relit-avatar render path (arXiv 2407.10707,
Sec. 3 and App. A-B), in plain C (avatar_oracle.c) and numpy / torch-CPU.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product package never imports, links or runs it,
and it shares no code with the CUDA path."""
