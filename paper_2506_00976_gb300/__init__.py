"""Certified quantization-based Wasserstein bounds on GB300 (placeholder; binding below)."""
