"""Batched evaluation of straight-line symbolic programs on GB300 (CusADi-style)."""
